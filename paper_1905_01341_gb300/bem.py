"""Python binding of libbem.so (include/bem.h): argument marshalling only.

Every function here has the name of the C entry point it calls and forwards plain
pointers and sizes; all arithmetic runs in the CUDA library. Arrays may be torch tensors
(CUDA or CPU) or numpy arrays; they must be contiguous and of the documented dtype. The
library must have been built (``paper_1905_01341_gb300.build.build()``); importing this
module without it raises, there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libbem.so")

BEM_OK = 0
BEM_ERR_ARG = 1
BEM_ERR_MESH = 2
BEM_ERR_NOT_BUILT = 3
BEM_ERR_NOCONV = 4
BEM_ERR_TIMEOUT = 5
BEM_ERR_CUDA = 6
BEM_ERR_NAN = 7
BEM_ERR_NOMEM = 8

BEM_PREC_FP64 = 0
BEM_PREC_MIXED = 1
BEM_MVP_FMM = 0
BEM_MVP_DIRECT = 1

EXPORTED = [
    "bem_params_default", "bem_create", "bem_destroy", "bem_set_stream", "bem_last_error",
    "bem_mesh_upload", "bem_points_upload", "bem_mesh_set_clusters", "bem_mesh_update_xyz", "fmm_build", "bem_apply", "bem_apply_sl",
    "bem_apply_dl", "bem_rhs", "bem_solve", "bem_precond_apply", "bem_get_geometry", "bem_get_stats",
    "bem_reset_stats", "bem_profile_enable", "bem_profile_read", "bem_phase_name",
    "bem_get_residual_history", "bem_step_params_default", "bem_step_init", "bem_step",
    "bem_step_get_state", "bem_step_set_state", "bem_step_filter", "bem_step_save", "bem_step_load", "bem_apply_direct_noalloc", "bem_mlp_init", "bem_mlp_set_mode", "bem_mlp_train",
    "bem_mlp_loss_grad", "bem_mlp_forward", "bem_mlp_get_params", "bem_mlp_set_params", "bem_mlp_info",
    "bem_m2l_orders", "bem_get_cluster_stats",
]

BEM_NUM_PHASES = 15


class bem_params(ctypes.Structure):
    _fields_ = [
        ("p_fmm", ctypes.c_int32),
        ("leaf_target", ctypes.c_int32),
        ("fixed_level", ctypes.c_int32),
        ("precision", ctypes.c_int32),
        ("mvp", ctypes.c_int32),
        ("diag_precision", ctypes.c_int32),
        ("diag_p_fmm", ctypes.c_int32),
        ("overlap", ctypes.c_int32),
        ("m2l_tensor_cores", ctypes.c_int32),
        ("gmres_precond", ctypes.c_int32),
        ("gmres_maxit", ctypes.c_int32),
        ("gmres_restart", ctypes.c_int32),
        ("gmres_tol", ctypes.c_double),
        ("m2l_stages", ctypes.c_int32),
        ("p2p_blocks_per_sm", ctypes.c_int32),
        ("m2l_order_margin", ctypes.c_int32),
        ("m2l_target_major", ctypes.c_int32),
    ]


class bem_stats(ctypes.Structure):
    _fields_ = [
        ("n_apply", ctypes.c_int64),
        ("n_apply_rhs", ctypes.c_int64),
        ("p2p_pairs", ctypes.c_int64),
        ("m2l_pairs", ctypes.c_int64),
        ("levels", ctypes.c_int32),
        ("leaves", ctypes.c_int32),
        ("last_iters", ctypes.c_int32),
        ("last_mvps", ctypes.c_int32),
        ("last_relres", ctypes.c_double),
        ("last_build_ms", ctypes.c_double),
        ("n_launches", ctypes.c_int64),
        ("m2l_stages", ctypes.c_int32),
        ("overlap", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("p2p_blocks_per_sm", ctypes.c_int32),
        ("m2l_macs", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class bem_step_params(ctypes.Structure):
    _fields_ = [
        ("sigma", ctypes.c_double),
        ("kappa", ctypes.c_double),
        ("pa", ctypes.c_double),
        ("omega", ctypes.c_double),
        ("courant", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("pf", ctypes.c_int32),
        ("guess", ctypes.c_int32),
        ("ab_order", ctypes.c_int32),
        ("corrector", ctypes.c_int32),
        ("rk_order", ctypes.c_int32),
    ]


class bem_step_stats(ctypes.Structure):
    _fields_ = [
        ("t", ctypes.c_double),
        ("dt", ctypes.c_double),
        ("rhs_calls", ctypes.c_int32),
        ("gmres_iters", ctypes.c_int32),
        ("mvps", ctypes.c_int32),
        ("nonconverged", ctypes.c_int32),
        ("max_relres", ctypes.c_double),
        ("steps", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class bem_mlp_summary(ctypes.Structure):
    _fields_ = [
        ("dims", ctypes.c_int32 * 5),
        ("overlap", ctypes.c_int32),
        ("num_params", ctypes.c_int64),
        ("samples", ctypes.c_int64),
        ("compared_solves", ctypes.c_int64),
        ("iters_guess", ctypes.c_int64),
        ("iters_fallback", ctypes.c_int64),
        ("res0_guess", ctypes.c_double),
        ("res0_fallback", ctypes.c_double),
    ]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "dims"}
        d["dims"] = list(self.dims)
        return d


class BemError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("bem status %d: %s" % (code, msg))
        self.code = code


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libbem.so. Raises when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libbem.so is not built (%s); run paper_1905_01341_gb300.build.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        sig = {
            "bem_params_default": ([ctypes.POINTER(bem_params)], ctypes.c_int),
            "bem_create": ([ctypes.POINTER(vp), ctypes.POINTER(bem_params), vp], ctypes.c_int),
            "bem_destroy": ([vp], None),
            "bem_set_stream": ([vp, vp], ctypes.c_int),
            "bem_last_error": ([vp], ctypes.c_char_p),
            "bem_mesh_upload": ([vp, i64, vp, i64, vp, i64, vp, vp], ctypes.c_int),
            "bem_mesh_update_xyz": ([vp, vp], ctypes.c_int),
            "bem_points_upload": ([vp, i64, vp], ctypes.c_int),
            "bem_mesh_set_clusters": ([vp, i64, vp], ctypes.c_int),
            "fmm_build": ([vp], ctypes.c_int),
            "bem_apply": ([vp, dbl, vp, dbl, vp, vp], ctypes.c_int),
            "bem_apply_sl": ([vp, vp, vp], ctypes.c_int),
            "bem_apply_dl": ([vp, vp, vp], ctypes.c_int),
            "bem_rhs": ([vp, vp, vp], ctypes.c_int),
            "bem_precond_apply": ([vp, vp, vp], ctypes.c_int),
            "bem_solve": ([vp, vp, vp, ctypes.POINTER(i32), ctypes.POINTER(dbl)], ctypes.c_int),
            "bem_get_geometry": ([vp, vp, vp, vp, vp], ctypes.c_int),
            "bem_get_stats": ([vp, ctypes.POINTER(bem_stats)], ctypes.c_int),
            "bem_reset_stats": ([vp], ctypes.c_int),
            "bem_profile_enable": ([vp, ctypes.c_int], ctypes.c_int),
            "bem_profile_read": ([vp, ctypes.POINTER(dbl), ctypes.POINTER(i64)], ctypes.c_int),
            "bem_phase_name": ([ctypes.c_int], ctypes.c_char_p),
            "bem_get_residual_history": ([vp, ctypes.POINTER(dbl), i32, ctypes.POINTER(i32)], ctypes.c_int),
            "bem_step_params_default": ([ctypes.POINTER(bem_step_params)], ctypes.c_int),
            "bem_step_init": ([vp, vp, vp, ctypes.POINTER(bem_step_params)], ctypes.c_int),
            "bem_step": ([vp, ctypes.POINTER(bem_step_stats)], ctypes.c_int),
            "bem_step_get_state": ([vp, vp, vp, vp, ctypes.POINTER(dbl)], ctypes.c_int),
            "bem_step_set_state": ([vp, vp, vp, vp], ctypes.c_int),
            "bem_step_filter": ([vp, vp, vp], ctypes.c_int),
            "bem_step_save": ([vp, vp, i64, ctypes.POINTER(i64)], ctypes.c_int),
            "bem_step_load": ([vp, vp, i64], ctypes.c_int),
            "bem_apply_direct_noalloc": ([i64, vp, vp, vp, vp, vp, dbl, vp, dbl, vp, vp, vp], ctypes.c_int),
            "bem_mlp_init": ([vp, i32, i32, ctypes.c_uint64], ctypes.c_int),
            "bem_mlp_set_mode": ([vp, i32, i32, i32], ctypes.c_int),
            "bem_mlp_train": ([vp, i32, i32, dbl, ctypes.POINTER(dbl)], ctypes.c_int),
            "bem_mlp_loss_grad": ([vp, i32, vp, vp, ctypes.POINTER(dbl), vp], ctypes.c_int),
            "bem_mlp_forward": ([vp, i32, vp, vp], ctypes.c_int),
            "bem_mlp_get_params": ([vp, vp], ctypes.c_int),
            "bem_mlp_set_params": ([vp, vp], ctypes.c_int),
            "bem_mlp_info": ([vp, ctypes.POINTER(bem_mlp_summary)], ctypes.c_int),
            "bem_m2l_orders": ([i32, i32, ctypes.POINTER(i32)], ctypes.c_int),
            "bem_get_cluster_stats": ([vp, i64, vp, vp, vp, ctypes.POINTER(dbl)], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _ptr(x, dtype=None):
    """Raw pointer of a contiguous torch tensor or numpy array (None stays None)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        if dtype is not None and x.dtype != np.dtype(dtype):
            raise TypeError("expected dtype %s, got %s" % (dtype, x.dtype))
        return ctypes.c_void_p(x.ctypes.data)
    import torch  # torch tensors: device memory comes from torch

    if isinstance(x, torch.Tensor):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        want = {np.float64: torch.float64, np.int32: torch.int32, np.int64: torch.int64}.get(dtype)
        if want is not None and x.dtype != want:
            raise TypeError("expected dtype %s, got %s" % (want, x.dtype))
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    raise TypeError("unsupported array type %r" % type(x))


def _check(ctx, rc: int):
    if rc != BEM_OK:
        msg = lib().bem_last_error(ctx)
        raise BemError(rc, msg.decode() if msg else "")


# ------------------------------------------------------------------ one wrapper per entry point


def bem_params_default(**overrides) -> bem_params:
    p = bem_params()
    lib().bem_params_default(ctypes.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def bem_create(params: bem_params | None = None, stream=None):
    """Create a context on the current device. `stream`: a torch.cuda.Stream, an int
    handle, or None (torch's current stream)."""
    if stream is None:
        import torch

        stream = torch.cuda.current_stream()
    handle = stream if isinstance(stream, int) else stream.cuda_stream
    ctx = ctypes.c_void_p()
    rc = lib().bem_create(ctypes.byref(ctx), ctypes.byref(params) if params is not None else None,
                          ctypes.c_void_p(handle))
    _check(None, rc)
    return ctx


def bem_destroy(ctx) -> None:
    lib().bem_destroy(ctx)


def bem_set_stream(ctx, stream) -> None:
    handle = stream if isinstance(stream, int) else stream.cuda_stream
    _check(ctx, lib().bem_set_stream(ctx, ctypes.c_void_p(handle)))


def bem_last_error(ctx) -> str:
    m = lib().bem_last_error(ctx)
    return m.decode() if m else ""


def bem_mesh_upload(ctx, N, xyz, T, tri, M, vert_off, tri_off) -> None:
    _check(ctx, lib().bem_mesh_upload(ctx, int(N), _ptr(xyz, np.float64), int(T), _ptr(tri, np.int32), int(M),
                                      _ptr(vert_off, np.int64), _ptr(tri_off, np.int64)))


def bem_points_upload(ctx, N, xyz) -> None:
    _check(ctx, lib().bem_points_upload(ctx, int(N), _ptr(xyz, np.float64)))


def bem_mesh_set_clusters(ctx, C, bubble_off) -> None:
    _check(ctx, lib().bem_mesh_set_clusters(ctx, int(C), _ptr(bubble_off, np.int64)))


def bem_mesh_update_xyz(ctx, xyz) -> None:
    _check(ctx, lib().bem_mesh_update_xyz(ctx, _ptr(xyz, np.float64)))


def fmm_build(ctx) -> None:
    _check(ctx, lib().fmm_build(ctx))


def bem_apply(ctx, f, xL, g, xM, out) -> None:
    _check(ctx, lib().bem_apply(ctx, float(f), _ptr(xL, np.float64), float(g), _ptr(xM, np.float64),
                                _ptr(out, np.float64)))


def bem_apply_sl(ctx, q, out) -> None:
    _check(ctx, lib().bem_apply_sl(ctx, _ptr(q, np.float64), _ptr(out, np.float64)))


def bem_apply_dl(ctx, phi, out) -> None:
    _check(ctx, lib().bem_apply_dl(ctx, _ptr(phi, np.float64), _ptr(out, np.float64)))


def bem_rhs(ctx, phi, b) -> None:
    _check(ctx, lib().bem_rhs(ctx, _ptr(phi, np.float64), _ptr(b, np.float64)))


def bem_precond_apply(ctx, y, z) -> None:
    _check(ctx, lib().bem_precond_apply(ctx, _ptr(y, np.float64), _ptr(z, np.float64)))


def bem_solve(ctx, phi, q_inout, raise_on_noconv: bool = True):
    """Returns (iterations, true relative residual); q_inout holds the solution."""
    it = ctypes.c_int32(0)
    rr = ctypes.c_double(0.0)
    rc = lib().bem_solve(ctx, _ptr(phi, np.float64), _ptr(q_inout, np.float64), ctypes.byref(it), ctypes.byref(rr))
    if rc == BEM_ERR_NOCONV and not raise_on_noconv:
        return int(it.value), float(rr.value)
    _check(ctx, rc)
    return int(it.value), float(rr.value)


def bem_get_geometry(ctx, s=None, n=None, ldiag=None, mdiag=None) -> None:
    _check(ctx, lib().bem_get_geometry(ctx, _ptr(s, np.float64), _ptr(n, np.float64), _ptr(ldiag, np.float64),
                                       _ptr(mdiag, np.float64)))


def bem_get_residual_history(ctx) -> list:
    cnt = ctypes.c_int32(0)
    _check(ctx, lib().bem_get_residual_history(ctx, None, 0, ctypes.byref(cnt)))
    buf = (ctypes.c_double * max(1, cnt.value))()
    _check(ctx, lib().bem_get_residual_history(ctx, buf, cnt.value, ctypes.byref(cnt)))
    return [float(buf[i]) for i in range(cnt.value)]


def bem_step_params_default(**overrides) -> bem_step_params:
    sp = bem_step_params()
    lib().bem_step_params_default(ctypes.byref(sp))
    for k, v in overrides.items():
        setattr(sp, k, v)
    return sp


def bem_step_init(ctx, phi0, sp: bem_step_params | None = None, q0=None) -> None:
    _check(ctx, lib().bem_step_init(ctx, _ptr(phi0, np.float64), _ptr(q0, np.float64),
                                    ctypes.byref(sp) if sp is not None else None))


def bem_step(ctx) -> dict:
    st = bem_step_stats()
    _check(ctx, lib().bem_step(ctx, ctypes.byref(st)))
    return st.as_dict()


def bem_step_get_state(ctx, xyz=None, phi=None, q=None) -> float:
    t = ctypes.c_double(0.0)
    _check(ctx, lib().bem_step_get_state(ctx, _ptr(xyz, np.float64), _ptr(phi, np.float64), _ptr(q, np.float64),
                                         ctypes.byref(t)))
    return float(t.value)


def bem_step_set_state(ctx, xyz=None, phi=None, q=None) -> None:
    _check(ctx, lib().bem_step_set_state(ctx, _ptr(xyz, np.float64), _ptr(phi, np.float64), _ptr(q, np.float64)))


def bem_step_filter(ctx, x, y) -> None:
    _check(ctx, lib().bem_step_filter(ctx, _ptr(x, np.float64), _ptr(y, np.float64)))


def bem_step_save(ctx, buf=None) -> int:
    """Write the time-integration checkpoint into `buf` (a uint8 numpy array or tensor of at
    least the returned size; None only queries the size). Returns the size in bytes."""
    size = ctypes.c_int64(0)
    _check(ctx, lib().bem_step_save(ctx, None, 0, ctypes.byref(size)))
    if buf is not None:
        nbytes = buf.nbytes if isinstance(buf, np.ndarray) else buf.numel() * buf.element_size()
        _check(ctx, lib().bem_step_save(ctx, _ptr(buf), int(nbytes), ctypes.byref(size)))
    return int(size.value)


def bem_step_load(ctx, buf) -> None:
    nbytes = buf.nbytes if isinstance(buf, np.ndarray) else buf.numel() * buf.element_size()
    _check(ctx, lib().bem_step_load(ctx, _ptr(buf), int(nbytes)))


def _noalloc_arg(name, x, count):
    """A float64 CUDA tensor of the current device with at least `count` elements: the C entry
    point takes raw device pointers and cannot check lengths."""
    import torch

    if not isinstance(x, torch.Tensor) or not x.is_cuda:
        raise BemError(BEM_ERR_ARG, "bem_apply_direct_noalloc: %s must be a CUDA tensor" % name)
    if x.device.index != torch.cuda.current_device():
        raise BemError(BEM_ERR_ARG, "bem_apply_direct_noalloc: %s is on another device" % name)
    if x.dtype != torch.float64 or not x.is_contiguous():
        raise BemError(BEM_ERR_ARG, "bem_apply_direct_noalloc: %s must be contiguous float64" % name)
    if x.numel() < count:
        raise BemError(BEM_ERR_ARG, "bem_apply_direct_noalloc: %s has %d elements, needs %d" % (name, x.numel(), count))
    return x


def bem_apply_direct_noalloc(N, xyz, s, n, ldiag, mdiag, f, xL, g, xM, out, stream=0) -> None:
    """Allocation-free direct product on caller-owned device arrays (see include/bem.h): every
    array a contiguous float64 CUDA tensor of the current device, xyz and n with 3N elements,
    the others with N (xL may be None when f == 0, xM when g == 0)."""
    N = int(N)
    for name, x, cnt in (("xyz", xyz, 3 * N), ("s", s, N), ("n", n, 3 * N), ("ldiag", ldiag, N),
                         ("mdiag", mdiag, N), ("out", out, N)):
        _noalloc_arg(name, x, cnt)
    if float(f) != 0.0:
        _noalloc_arg("xL", xL, N)
    if float(g) != 0.0:
        _noalloc_arg("xM", xM, N)
    handle = stream if isinstance(stream, int) else stream.cuda_stream
    rc = lib().bem_apply_direct_noalloc(N, _ptr(xyz, np.float64), _ptr(s, np.float64), _ptr(n, np.float64),
                                        _ptr(ldiag, np.float64), _ptr(mdiag, np.float64), float(f),
                                        _ptr(xL, np.float64), float(g), _ptr(xM, np.float64),
                                        _ptr(out, np.float64), ctypes.c_void_p(handle))
    _check(None, rc)


def bem_mlp_init(ctx, hidden=256, lmax=10, seed=0) -> None:
    _check(ctx, lib().bem_mlp_init(ctx, int(hidden), int(lmax), int(seed)))


def bem_mlp_set_mode(ctx, record=False, use_guess=False, compare=False) -> None:
    _check(ctx, lib().bem_mlp_set_mode(ctx, int(bool(record)), int(bool(use_guess)), int(bool(compare))))


def bem_mlp_train(ctx, epochs, batch, lr) -> float:
    loss = ctypes.c_double(0.0)
    _check(ctx, lib().bem_mlp_train(ctx, int(epochs), int(batch), float(lr), ctypes.byref(loss)))
    return float(loss.value)


def bem_mlp_loss_grad(ctx, F, T, grads):
    """F [B, d_in], T [B, d_out] (float64); grads [num_params] receives the gradient."""
    loss = ctypes.c_double(0.0)
    _check(ctx, lib().bem_mlp_loss_grad(ctx, int(F.shape[0]), _ptr(F, np.float64), _ptr(T, np.float64),
                                        ctypes.byref(loss), _ptr(grads, np.float64)))
    return float(loss.value)


def bem_mlp_forward(ctx, F, Y) -> None:
    _check(ctx, lib().bem_mlp_forward(ctx, int(F.shape[0]), _ptr(F, np.float64), _ptr(Y, np.float64)))


def bem_mlp_get_params(ctx, out) -> None:
    _check(ctx, lib().bem_mlp_get_params(ctx, _ptr(out, np.float64)))


def bem_mlp_set_params(ctx, params) -> None:
    _check(ctx, lib().bem_mlp_set_params(ctx, _ptr(params, np.float64)))


def bem_mlp_info(ctx) -> dict:
    st = bem_mlp_summary()
    _check(ctx, lib().bem_mlp_info(ctx, ctypes.byref(st)))
    return st.as_dict()


def bem_get_cluster_stats(ctx, C) -> dict:
    """Per-cluster GMRES iterations, true relative residuals and device ms until final of the
    last clustered solve, and that solve's device ms."""
    it = np.zeros(C, np.int32)
    rr = np.zeros(C)
    ms = np.zeros(C)
    sm = ctypes.c_double(0.0)
    _check(ctx, lib().bem_get_cluster_stats(ctx, int(C), _ptr(it), _ptr(rr), _ptr(ms), ctypes.byref(sm)))
    return {"iters": it, "relres": rr, "done_ms": ms, "solve_ms": float(sm.value)}


def bem_m2l_orders(p_fmm: int, margin: int) -> list:
    """Truncation order of each M2L offset class (316, lexicographic offsets)."""
    out = (ctypes.c_int32 * 316)()
    rc = lib().bem_m2l_orders(int(p_fmm), int(margin), out)
    if rc != BEM_OK:
        raise BemError(rc, "bad p_fmm or margin")
    return [int(v) for v in out]


def bem_get_stats(ctx) -> dict:
    st = bem_stats()
    _check(ctx, lib().bem_get_stats(ctx, ctypes.byref(st)))
    return st.as_dict()


def bem_reset_stats(ctx) -> None:
    _check(ctx, lib().bem_reset_stats(ctx))


def bem_profile_enable(ctx, on: bool = True) -> None:
    _check(ctx, lib().bem_profile_enable(ctx, 1 if on else 0))


def bem_profile_read(ctx) -> dict:
    """{phase name: (device ms, timed intervals)} since the last read."""
    ms = (ctypes.c_double * BEM_NUM_PHASES)()
    cnt = (ctypes.c_int64 * BEM_NUM_PHASES)()
    _check(ctx, lib().bem_profile_read(ctx, ms, cnt))
    return {bem_phase_name(i): (float(ms[i]), int(cnt[i])) for i in range(BEM_NUM_PHASES)}


def bem_phase_name(i: int) -> str:
    n = lib().bem_phase_name(int(i))
    return n.decode() if n else ""


# ------------------------------------------------------------------ convenience


class BemContext:
    """Owns one context; methods take torch tensors or numpy arrays (SoA layouts of bem.h)."""

    def __init__(self, stream=None, **params):
        self.params = bem_params_default(**params)
        self.ctx = bem_create(self.params, stream)
        self.N = 0

    def close(self):
        if self.ctx is not None:
            bem_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def upload(self, xyz_soa, tri_soa, vert_off, tri_off):
        N = int(xyz_soa.shape[-1])
        T = int(tri_soa.shape[-1])
        M = int(vert_off.shape[0]) - 1
        bem_mesh_upload(self.ctx, N, xyz_soa, T, tri_soa, M, vert_off, tri_off)
        self.N = N

    def upload_mesh(self, mesh):
        """Upload a synth.Mesh-like object (numpy arrays) from host memory."""
        self.upload(mesh.xyz_soa(), mesh.tri_soa(), np.ascontiguousarray(mesh.vert_off, np.int64),
                    np.ascontiguousarray(mesh.tri_off, np.int64))

    def build(self):
        fmm_build(self.ctx)

    def apply(self, f, xL, g, xM, out):
        bem_apply(self.ctx, f, xL, g, xM, out)
        return out

    def solve(self, phi, q, raise_on_noconv=True):
        return bem_solve(self.ctx, phi, q, raise_on_noconv)

    def precond_apply(self, y, z):
        bem_precond_apply(self.ctx, y, z)

    def stats(self) -> dict:
        return bem_get_stats(self.ctx)

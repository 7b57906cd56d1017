"""CPU FP64 oracle for the FMM-accelerated boundary-element method of arXiv:1905.01341.

TEST INFRASTRUCTURE. Only the tests, the package smoke check and the benchmark's
CPU-baseline leg may import this package. The product path (the CUDA library and its
Python binding) never imports or calls it, and the two share no code.

The oracle is the plain dense discrete operator the FMM approximates, written out step
by step in the paper's notation:
  * `vertex_geometry`  — Eq. (ns1): s_j, n_j from triangle areas and normals.
  * `offdiag_apply`    — Eq. (ns1)/(2.13)/(3.27): f L_off xL + g M_off xM, j != i.
  * `diagonals`        — Section 3.3, Eqs. (s3) and (s5): singular diagonals from the
                          integral identities with test functions 1, x, y, z.
  * `BemOperator`      — Eq. (3.1)/(3.2): L q, M phi, right-hand side b.
  * `gmres`            — Section 3.8: unpreconditioned GMRES (Saad-Schultz), modified
                          Gram-Schmidt Arnoldi and Givens rotations, initial guess x0.
  * `solve`            — Eq. (3.2): given phi on S, return q = dphi/dn.
  * `rayleigh_plesset` — Eq. (4.1): radius history of a spherical bubble (see rp.py).
Large meshes use the paper's own checkpoint method (Section 3.9): the direct sum at a
random sample of receivers.
"""
from __future__ import annotations

import ctypes
import math

import numpy as np

from . import build as _build
from .gmres import gmres  # noqa: F401  (re-exported)

_LIB = None


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        lib.oracle_vertex_geometry.argtypes = [ctypes.c_int64, dp, ctypes.c_int64,
                                               ctypes.POINTER(ctypes.c_int32), dp, dp]
        lib.oracle_vertex_geometry.restype = ctypes.c_int
        lib.oracle_offdiag_apply.argtypes = [ctypes.c_int64, dp, dp, dp, ctypes.c_double, dp,
                                             ctypes.c_double, dp, ctypes.c_int64,
                                             ctypes.POINTER(ctypes.c_int64), dp]
        lib.oracle_offdiag_apply.restype = None
        lib.oracle_offdiag_dense.argtypes = [ctypes.c_int64, dp, dp, dp, dp, dp]
        lib.oracle_offdiag_dense.restype = None
        lib.oracle_num_threads.argtypes = []
        lib.oracle_num_threads.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    """OpenMP threads the direct sums run on."""
    return int(_lib().oracle_num_threads())


def vertex_geometry(xyz: np.ndarray, tri: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Eq. (ns1): vertex weights s [N] and unit normals n [N, 3]."""
    xyz = _c(xyz, np.float64)
    tri = _c(tri, np.int32)
    n = xyz.shape[0]
    s = np.empty(n)
    nrm = np.empty((n, 3))
    rc = _lib().oracle_vertex_geometry(n, _dp(xyz), tri.shape[0],
                                       tri.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                       _dp(s), _dp(nrm))
    if rc != 0:
        raise ValueError("invalid mesh (oracle_vertex_geometry returned %d)" % rc)
    return s, nrm


def offdiag_apply(xyz, s, nrm, f, xL, g, xM, recv=None) -> np.ndarray:
    """Eq. (ns1)/(3.27): out_i = f sum_{j!=i} L_ij xL_j + g sum_{j!=i} M_ij xM_j for the
    receivers `recv` (all vertices when None)."""
    xyz = _c(xyz, np.float64)
    s = _c(s, np.float64)
    nrm = _c(nrm, np.float64)
    xL = None if (f == 0.0 or xL is None) else _c(xL, np.float64)
    xM = None if (g == 0.0 or xM is None) else _c(xM, np.float64)
    n = xyz.shape[0]
    if recv is None:
        out = np.empty(n)
        _lib().oracle_offdiag_apply(n, _dp(xyz), _dp(s), _dp(nrm), float(f), _dp(xL), float(g),
                                    _dp(xM), n, None, _dp(out))
    else:
        recv = _c(recv, np.int64)
        out = np.empty(recv.shape[0])
        _lib().oracle_offdiag_apply(n, _dp(xyz), _dp(s), _dp(nrm), float(f), _dp(xL), float(g),
                                    _dp(xM), recv.shape[0],
                                    recv.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(out))
    return out


def offdiag_dense(xyz, s, nrm) -> tuple[np.ndarray, np.ndarray]:
    """Eq. (ns1): the dense off-diagonal N x N matrices (L_off, M_off); small N only."""
    xyz = _c(xyz, np.float64)
    n = xyz.shape[0]
    L = np.empty((n, n))
    M = np.empty((n, n))
    _lib().oracle_offdiag_dense(n, _dp(xyz), _dp(_c(s, np.float64)), _dp(_c(nrm, np.float64)),
                                _dp(L), _dp(M))
    return L, M


def diagonals(xyz, s, nrm, recv=None) -> tuple[np.ndarray, np.ndarray]:
    """Section 3.3: singular diagonal elements from the integral identities.

    Eq. (s3) (test function Phi = 1, Q = 0):  M_ii = -1/2 - sum_{j!=i} M_ij.
    Eq. (s5) (Phi = x, y, z; Q = n_x, n_y, n_z):
        L_ii = n_i . [ sum_{j!=i} (M_ij r_j - L_ij n_j) + (1/2 + M_ii) r_i ].
    The sums run over all vertices of all bubbles. Four off-diagonal applications, as the
    paper counts them (one for M_ii, three for L_ii). Returns (Ldiag, Mdiag) at `recv`.
    """
    xyz = _c(xyz, np.float64)
    ones = np.ones(xyz.shape[0])
    mdiag = -0.5 - offdiag_apply(xyz, s, nrm, 0.0, None, 1.0, ones, recv)
    ri = xyz if recv is None else xyz[recv]
    ni = nrm if recv is None else nrm[recv]
    ldiag = np.zeros_like(mdiag)
    for c in range(3):
        # sum_{j!=i} (M_ij r_j,c - L_ij n_j,c): f = -1 on the single layer with X = n_c,
        # g = +1 on the double layer with X = r_c.
        vc = offdiag_apply(xyz, s, nrm, -1.0, nrm[:, c], 1.0, xyz[:, c], recv)
        ldiag += ni[:, c] * (vc + (0.5 + mdiag) * ri[:, c])
    return ldiag, mdiag


class BemOperator:
    """The discrete operators of Eq. (3.2) on one mesh: L = L_off + diag(Ldiag) and
    M = M_off + diag(Mdiag), with geometry from Eq. (ns1) and diagonals from Section 3.3."""

    def __init__(self, xyz: np.ndarray, tri: np.ndarray):
        self.xyz = _c(xyz, np.float64)
        self.tri = _c(tri, np.int32)
        self.s, self.n = vertex_geometry(self.xyz, self.tri)
        self.ldiag, self.mdiag = diagonals(self.xyz, self.s, self.n)
        self.n_apply = 0

    @property
    def size(self) -> int:
        return self.xyz.shape[0]

    def apply(self, f, xL, g, xM, recv=None) -> np.ndarray:
        """Eq. (3.27): (f L + g M) applied with separate inputs for the two layers."""
        self.n_apply += 1
        out = offdiag_apply(self.xyz, self.s, self.n, f, xL, g, xM, recv)
        idx = slice(None) if recv is None else recv
        if f != 0.0:
            out = out + f * self.ldiag[idx] * np.asarray(xL)[idx]
        if g != 0.0:
            out = out + g * self.mdiag[idx] * np.asarray(xM)[idx]
        return out

    def apply_L(self, q, recv=None) -> np.ndarray:
        return self.apply(1.0, q, 0.0, None, recv)

    def apply_M(self, phi, recv=None) -> np.ndarray:
        return self.apply(0.0, None, 1.0, phi, recv)

    def rhs(self, phi) -> np.ndarray:
        """Eq. (3.1): b = -phi/2 + M phi."""
        return -0.5 * np.asarray(phi) + self.apply_M(phi)

    def dense(self) -> tuple[np.ndarray, np.ndarray]:
        """Assembled L and M (small N): off-diagonal matrices plus the identity diagonals."""
        L, M = offdiag_dense(self.xyz, self.s, self.n)
        L[np.diag_indices_from(L)] = self.ldiag
        M[np.diag_indices_from(M)] = self.mdiag
        return L, M


def solve(op: BemOperator, phi, q0=None, tol: float = 1e-10, maxit: int = 100, restart=None):
    """Eq. (3.2): solve L q = b, b = -phi/2 + M phi, by unpreconditioned GMRES with initial
    guess q0 (zero when None). Returns (q, iterations, true relative residual, MVPs)."""
    b = op.rhs(phi)
    x0 = np.zeros_like(b) if q0 is None else np.asarray(q0, dtype=np.float64)
    return gmres(op.apply_L, b, x0, tol=tol, maxit=maxit, restart=restart)


def checkpoint_receivers(n: int, count: int, seed: int) -> np.ndarray:
    """Sorted random sample of `count` distinct receivers (Section 3.9 uses sqrt(N) of them)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.sort(rng.choice(n, size=min(count, n), replace=False)).astype(np.int64)


def sqrt_n(n: int) -> int:
    return int(math.isqrt(n))

"""The allocation-free direct product (bem_apply_direct_noalloc) against the context-based
direct product (bem_apply, BEM_MVP_DIRECT + BEM_PREC_MIXED).

Callers that cannot allocate device memory at call time (a fixed memory pool owned by another
framework, a latency-critical loop) use the allocation-free entry point; it must give the same
result as the regular path. This file is collected last so that a failure here does not hide
the other tests, and it runs on its own too.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def test_noalloc_direct_product_matches_context_product_twice():
    from paper_1905_01341_gb300 import bem, build

    build.build()
    rng = np.random.Generator(np.random.PCG64(21))
    radii = np.array([1.0, 0.7, 1.2])
    centres = np.array([[0.0, 0.0, 0.0], [2.5, 0.3, 0.0], [-0.2, 3.1, 0.4]])
    mesh = synth.cluster(3, radii, centres)  # 1926 vertices: several tiles and a ragged one
    N = mesh.n
    ctx = bem.BemContext(mvp=bem.BEM_MVP_DIRECT, precision=bem.BEM_PREC_MIXED)
    ctx.upload(torch.from_numpy(mesh.xyz_soa()).cuda(), torch.from_numpy(mesh.tri_soa()).cuda(),
               torch.from_numpy(mesh.vert_off).cuda(), torch.from_numpy(mesh.tri_off).cuda())
    ctx.build()
    s = torch.empty(N, dtype=torch.float64, device="cuda")
    n = torch.empty(3 * N, dtype=torch.float64, device="cuda")
    ld = torch.empty(N, dtype=torch.float64, device="cuda")
    md = torch.empty(N, dtype=torch.float64, device="cuda")
    bem.bem_get_geometry(ctx.ctx, s, n, ld, md)
    xyz = torch.from_numpy(mesh.xyz_soa()).cuda().reshape(-1)
    stream = torch.cuda.current_stream()
    for f, g in ((0.7, -1.3), (1.0, 0.0)):  # two calls in a row, different inputs
        xL = torch.from_numpy(rng.standard_normal(N)).cuda()
        xM = torch.from_numpy(rng.standard_normal(N)).cuda()
        ref = torch.empty(N, dtype=torch.float64, device="cuda")
        ctx.apply(f, xL, g, xM, ref)
        out = torch.full((N,), np.nan, dtype=torch.float64, device="cuda")
        bem.bem_apply_direct_noalloc(N, xyz, s, n, ld, md, f, xL, g, xM, out, stream)
        torch.cuda.synchronize()
        assert rel(out.cpu().numpy(), ref.cpu().numpy()) <= 1e-12
    # sizes beyond the fixed scratch are rejected by the C entry point with a clear error,
    # before any pointer is used
    P = lambda t: ctypes.c_void_p(t.data_ptr())  # noqa: E731
    rc = bem.lib().bem_apply_direct_noalloc(262145, P(xyz), P(s), P(n), P(ld), P(md), 1.0, P(xL), 0.0, None,
                                            P(out), ctypes.c_void_p(stream.cuda_stream))
    assert rc == bem.BEM_ERR_ARG and "262144" in bem.bem_last_error(None)
    # a host array is rejected by the C entry point (nothing is launched)
    host = np.zeros(N)
    rc = bem.lib().bem_apply_direct_noalloc(N, P(xyz), P(s), P(n), P(ld), P(md), 1.0,
                                            ctypes.c_void_p(host.ctypes.data), 0.0, None, P(out),
                                            ctypes.c_void_p(stream.cuda_stream))
    assert rc == bem.BEM_ERR_ARG and "xL" in bem.bem_last_error(None)
    # and by the binding, as are short tensors
    with pytest.raises(bem.BemError):
        bem.bem_apply_direct_noalloc(N, xyz, s, n, ld, md, 1.0, host, 0.0, None, out, stream)
    with pytest.raises(bem.BemError):
        bem.bem_apply_direct_noalloc(N, xyz[:N], s, n, ld, md, 1.0, xL, 0.0, None, out, stream)
    ctx.close()


def test_noalloc_at_the_largest_accepted_size():
    """N = 262144 fills the whole scratch array (hi and lo of all three coordinates). Free
    points (unit weights, normals along z, zero diagonals) against the context's direct FP32
    product of the same points: the same kernels on the same inputs. Also the single-layer-only
    call with a null double-layer input."""
    from paper_1905_01341_gb300 import bem, build

    build.build()
    N = 262144
    pts, _ = synth.random_cube_points(N, seed=23)
    xyz = torch.from_numpy(np.ascontiguousarray(pts.T)).cuda()
    ctx = bem.BemContext(mvp=bem.BEM_MVP_DIRECT, precision=bem.BEM_PREC_MIXED)
    bem.bem_points_upload(ctx.ctx, N, xyz)
    ctx.build()
    s = torch.ones(N, dtype=torch.float64, device="cuda")
    n = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    n[2 * N:] = 1.0
    zero = torch.zeros(N, dtype=torch.float64, device="cuda")
    rng = np.random.Generator(np.random.PCG64(24))
    stream = torch.cuda.current_stream()
    flat = xyz.reshape(-1)
    for f, g in ((1.0, 0.0), (0.4, 2.5)):
        xL = torch.from_numpy(rng.standard_normal(N)).cuda()
        xM = torch.from_numpy(rng.standard_normal(N)).cuda() if g != 0.0 else None
        ref = torch.empty(N, dtype=torch.float64, device="cuda")
        ctx.apply(f, xL, g, xM, ref)
        out = torch.full((N,), np.nan, dtype=torch.float64, device="cuda")
        bem.bem_apply_direct_noalloc(N, flat, s, n, zero, zero, f, xL, g, xM, out, stream)
        torch.cuda.synchronize()
        o, r = out.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(o).all()
        assert rel(o, r) <= 1e-12
    ctx.close()

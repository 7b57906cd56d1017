"""The allocation-free direct product (bem_apply_direct_noalloc) against the context-based
direct product (bem_apply, BEM_MVP_DIRECT + BEM_PREC_MIXED).

Callers that cannot allocate device memory at call time (a fixed memory pool owned by another
framework, a latency-critical loop) use the allocation-free entry point; it must give the same
result as the regular path. This file is collected last so that a failure here does not hide
the other tests, and it runs on its own too.
"""
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
    # sizes beyond the fixed scratch are rejected with a clear error
    with pytest.raises(bem.BemError) as e:
        bem.bem_apply_direct_noalloc(262145, xyz, s, n, ld, md, 1.0, xL, 0.0, None, out, stream)
    assert e.value.code == bem.BEM_ERR_ARG and "262144" in str(e.value)
    ctx.close()

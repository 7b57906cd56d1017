"""The 3.21M-unknown cluster (5000 icosphere-L3 bubbles, the benchmark's workload) in the
configuration the benchmark times (mixed precision, p = 14, autotuned depth): the products and
the identity diagonals agree with the oracle's direct FP64 sums at sampled receivers."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.fixture(scope="module")
def fullsize():
    mesh, phi = synth.workload_cluster(bubbles=5000, level=3, seed=3)
    s, n = oracle.vertex_geometry(mesh.xyz, mesh.tri)
    recv = oracle.checkpoint_receivers(mesh.n, 400, 17)
    ld, md = oracle.diagonals(mesh.xyz, s, n, recv)
    rng = np.random.Generator(np.random.PCG64(18))
    x = rng.standard_normal(mesh.n)
    offL = oracle.offdiag_apply(mesh.xyz, s, n, 1.0, x, 0.0, None, recv)
    offM = oracle.offdiag_apply(mesh.xyz, s, n, 0.0, None, 1.0, phi, recv)
    return mesh, phi, x, recv, ld, md, offL + ld * x[recv], offM + md * phi[recv]


def test_fullsize_cluster_products_and_diagonals_at_sampled_receivers(fullsize):
    from paper_1905_01341_gb300 import bem

    mesh, phi, x, recv, ld, md, eL, eM = fullsize
    ctx = bem.BemContext(mvp=bem.BEM_MVP_FMM, precision=bem.BEM_PREC_MIXED, p_fmm=14, leaf_target=0)
    ctx.upload_mesh(mesh)
    ctx.build()
    N = mesh.n
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    s = torch.zeros(N, dtype=torch.float64, device="cuda")
    n = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    gl = torch.zeros_like(s)
    gm = torch.zeros_like(s)
    bem.bem_get_geometry(ctx.ctx, s, n, gl, gm)
    o1 = torch.zeros_like(s)
    o2 = torch.zeros_like(s)
    ctx.apply(1.0, dev(x), 0.0, None, o1)
    ctx.apply(0.0, None, 1.0, dev(phi), o2)
    gl, gm = gl.cpu().numpy()[recv], gm.cpu().numpy()[recv]
    errs = {"L": rel(o1.cpu().numpy()[recv], eL), "M": rel(o2.cpu().numpy()[recv], eM),
            "Ldiag": rel(gl, ld), "Mdiag": rel(gm, md)}
    print("full-size errors at 400 receivers:", {k: "%.2e" % v for k, v in errs.items()},
          "levels", ctx.stats()["levels"])
    ctx.close()
    assert errs["L"] < 1e-5 and errs["M"] < 1e-5

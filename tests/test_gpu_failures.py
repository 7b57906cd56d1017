"""Failure reporting of the C ABI, triggered from the host with valid device work only: a
GMRES limit that cannot be met returns BEM_ERR_NOCONV with the last iterate and its true
residual, and a non-finite coordinate is reported as BEM_ERR_NAN by fmm_build before any
geometry or octree is formed from it."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _bem():
    from paper_1905_01341_gb300 import bem

    return bem


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1905_01341_gb300 import build

    build.build()


def _ctx(mesh, **params):
    bem = _bem()
    ctx = bem.BemContext(**params)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
    ctx.upload(d(mesh.xyz_soa()), d(mesh.tri_soa()), d(mesh.vert_off), d(mesh.tri_off))
    return ctx


@pytest.mark.parametrize("maxit", [1, 3])
def test_gmres_iteration_limit_returns_noconv_with_the_last_iterate(maxit):
    bem = _bem()
    mesh, phi = synth.workload_single_sphere()
    ctx = _ctx(mesh, mvp=bem.BEM_MVP_DIRECT, precision=bem.BEM_PREC_FP64, gmres_tol=1e-12, gmres_maxit=maxit)
    ctx.build()
    q = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
    with pytest.raises(bem.BemError) as ei:
        ctx.solve(torch.from_numpy(phi).cuda(), q)
    assert ei.value.code == bem.BEM_ERR_NOCONV
    # the same call without raising reports the iterations and the true residual of q
    q.zero_()
    it, rr = ctx.solve(torch.from_numpy(phi).cuda(), q, raise_on_noconv=False)
    assert it == maxit and 1e-12 < rr < 1.0
    st = ctx.stats()
    assert st["last_iters"] == maxit and st["last_relres"] == rr
    # q is the last iterate: its residual against the oracle's operator is the reported one
    op = oracle.BemOperator(mesh.xyz, mesh.tri)
    b = op.rhs(phi)
    qh = q.cpu().numpy()
    assert np.linalg.norm(qh) > 0.0
    true = np.linalg.norm(b - op.apply_L(qh)) / np.linalg.norm(b)
    assert abs(true - rr) <= 1e-9 * max(1.0, rr) + 1e-12
    ctx.close()


@pytest.mark.parametrize("where", ["mesh", "points"])
def test_nonfinite_coordinate_returns_nan_status(where):
    bem = _bem()
    mesh, _ = synth.workload_single_sphere()
    bad = mesh.xyz_soa().copy()
    bad[1, 17] = np.nan
    if where == "mesh":
        ctx = bem.BemContext(p_fmm=8, fixed_level=3)
        d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()  # noqa: E731
        ctx.upload(d(bad), d(mesh.tri_soa()), d(mesh.vert_off), d(mesh.tri_off))
    else:
        ctx = bem.BemContext(p_fmm=8, fixed_level=3)
        bem.bem_points_upload(ctx.ctx, mesh.n, torch.from_numpy(bad).cuda())
    with pytest.raises(bem.BemError) as ei:
        ctx.build()
    assert ei.value.code == bem.BEM_ERR_NAN
    assert "non-finite" in bem.bem_last_error(ctx.ctx)
    # the context stays usable: a finite mesh builds and applies afterwards
    xs = torch.from_numpy(np.ascontiguousarray(mesh.xyz_soa())).cuda()
    if where == "mesh":
        bem.bem_mesh_update_xyz(ctx.ctx, xs)
    else:
        bem.bem_points_upload(ctx.ctx, mesh.n, xs)
    ctx.build()
    out = torch.empty(mesh.n, dtype=torch.float64, device="cuda")
    ctx.apply(1.0, torch.ones(mesh.n, dtype=torch.float64, device="cuda"), 0.0, None, out)
    assert torch.isfinite(out).all()
    ctx.close()

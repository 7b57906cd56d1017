"""Independent clusters stepped together (bem_mesh_set_clusters): one octree cube per cluster,
no interaction across clusters, one launch per phase for all of them. The products and solves
equal the oracle's taken cluster by cluster."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _clusters():
    rng = np.random.Generator(np.random.PCG64(41))
    parts = []
    for nb, lev in ((1, 3), (5, 2), (9, 3), (3, 4)):  # uneven sizes and mesh levels
        radii = np.exp(0.3 * rng.standard_normal(nb))
        box = max(4.0 * nb ** (1 / 3), 4.0 * radii.max())
        centres = synth._place_centres(radii, box, 0.5, rng) + rng.standard_normal(3) * 0.5
        parts.append(synth.cluster(lev, radii, centres))
    # clusters overlap in space on purpose: only the cluster split keeps them apart
    xyz = np.concatenate([m.xyz for m in parts])
    tris, voff, toff, boff = [], [0], [0], [0]
    for m in parts:
        tris.append(m.tri + voff[-1])
        for b in range(m.m):
            voff.append(voff[-1] + int(m.vert_off[b + 1] - m.vert_off[b]))
            toff.append(toff[-1] + int(m.tri_off[b + 1] - m.tri_off[b]))
        boff.append(boff[-1] + m.m)
    mesh = synth.Mesh(xyz=xyz, tri=np.concatenate(tris).astype(np.int32), vert_off=np.array(voff, np.int64),
                      tri_off=np.array(toff, np.int64), centres=np.zeros((boff[-1], 3)), radii=np.ones(boff[-1]))
    return mesh, parts, np.array(boff, np.int64)


# The GMRES target of the mixed path is 1e-7: its products round in FP32, so they are linear
# only to about that level and the true residual stops falling there.
@pytest.mark.parametrize("prec,p,tol,gtol", [(0, 18, 1e-6, 1e-9), (1, 14, 1e-5, 1e-7)])
def test_cluster_products_and_solve_match_separate_oracles(prec, p, tol, gtol):
    from paper_1905_01341_gb300 import bem

    mesh, parts, boff = _clusters()
    ctx = bem.BemContext(mvp=bem.BEM_MVP_FMM, precision=prec, p_fmm=p, leaf_target=32, gmres_tol=gtol,
                         gmres_maxit=400, gmres_restart=100)
    ctx.upload_mesh(mesh)
    bem.bem_mesh_set_clusters(ctx.ctx, len(parts), boff)
    ctx.build()
    rng = np.random.Generator(np.random.PCG64(42))
    xL, xM = rng.standard_normal(mesh.n), rng.standard_normal(mesh.n)
    out = np.zeros(mesh.n)
    ctx.apply(0.7, xL, -1.3, xM, out)
    refs, a = [], 0
    for m in parts:
        op = oracle.BemOperator(m.xyz, m.tri)
        refs.append(op.apply(0.7, xL[a:a + m.n], -1.3, xM[a:a + m.n]))
        a += m.n
    assert rel(out, np.concatenate(refs)) < tol
    # solve: the joint system is block-diagonal
    phi = rng.standard_normal(mesh.n) * 0.1 + 1.0
    q = np.zeros(mesh.n)
    it, rr = ctx.solve(phi, q)
    assert rr <= gtol
    qr, a = [], 0
    for m in parts:
        op = oracle.BemOperator(m.xyz, m.tri)
        qq, _, _, _ = oracle.solve(op, phi[a:a + m.n], tol=1e-11, maxit=300, restart=100)
        qr.append(qq)
        a += m.n
    assert rel(q, np.concatenate(qr)) < 50 * tol
    # every cluster met the tolerance on its own system, and its solution matches its oracle
    cs = bem.bem_get_cluster_stats(ctx.ctx, len(parts))
    assert np.all(cs["relres"] <= gtol) and np.all(cs["iters"] >= 1) and np.all(cs["iters"] <= it)
    assert np.all(cs["done_ms"] > 0) and np.all(cs["done_ms"] <= cs["solve_ms"] + 1e-6)
    a = 0
    for m, qq in zip(parts, qr):
        assert rel(q[a:a + m.n], qq) < 50 * tol
        a += m.n
    ctx.close()


def test_each_cluster_meets_its_own_tolerance():
    """One cluster's right-hand side is 1e-4 of the others': a single Krylov space over the
    stacked system stops on the global residual and would leave it far from converged; the
    per-cluster solves stop on each cluster's own residual: every cluster's solution has a small
    true residual against its own oracle operator."""
    from paper_1905_01341_gb300 import bem

    mesh, parts, boff = _clusters()
    ctx = bem.BemContext(mvp=bem.BEM_MVP_FMM, precision=0, p_fmm=18, leaf_target=32, gmres_tol=1e-8,
                         gmres_maxit=400, gmres_restart=100, gmres_precond=2)
    ctx.upload_mesh(mesh)
    bem.bem_mesh_set_clusters(ctx.ctx, len(parts), boff)
    ctx.build()
    rng = np.random.Generator(np.random.PCG64(43))
    phi = rng.standard_normal(mesh.n) * 0.1 + 1.0
    a0, a1 = parts[0].n, parts[0].n + parts[1].n
    phi[a0:a1] *= 1e-4  # the second cluster
    q = np.zeros(mesh.n)
    it, rr = ctx.solve(phi, q)
    cs = bem.bem_get_cluster_stats(ctx.ctx, len(parts))
    print("per-cluster iterations", cs["iters"], "relres", ["%.1e" % v for v in cs["relres"]],
          "done ms", ["%.2f" % v for v in cs["done_ms"]], "solve ms %.2f" % cs["solve_ms"])
    assert np.all(cs["relres"] <= 1e-8)
    a = 0
    for m in parts:
        op = oracle.BemOperator(m.xyz, m.tri)
        b = op.rhs(phi[a:a + m.n])
        true = np.linalg.norm(b - op.apply_L(q[a:a + m.n])) / np.linalg.norm(b)
        assert true < 2e-6  # the FP64 FMM operator at p = 18 is within ~1e-6 of the oracle's
        a += m.n
    ctx.close()


def test_clusters_need_the_fmm():
    from paper_1905_01341_gb300 import bem

    mesh, parts, boff = _clusters()
    ctx = bem.BemContext(mvp=bem.BEM_MVP_DIRECT)
    ctx.upload_mesh(mesh)
    bem.bem_mesh_set_clusters(ctx.ctx, len(parts), boff)
    with pytest.raises(bem.BemError) as e:
        ctx.build()
    assert e.value.code == bem.BEM_ERR_ARG
    ctx.close()

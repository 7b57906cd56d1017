"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Tolerances (relative L2 over all outputs): the FP64 direct path agrees with the oracle to
rounding (1e-11); the FP64 FMM path at p_fmm >= 14 within 1e-6 and the mixed-precision path
(FP32 near field and expansions) within 1e-5, the bounds set for the two paths.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _bem():
    from paper_1905_01341_gb300 import bem

    return bem


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def dev(x, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def make_ctx(mesh, **params):
    bem = _bem()
    ctx = bem.BemContext(**params)
    ctx.upload(dev(mesh.xyz_soa()), dev(mesh.tri_soa()), dev(mesh.vert_off), dev(mesh.tri_off))
    ctx.build()
    return ctx


def small_cluster(nb=3, level=3, seed=7):
    rng = np.random.Generator(np.random.PCG64(seed))
    radii = np.exp(0.3 * rng.standard_normal(nb))
    box = max(4.0 * nb ** (1 / 3), 4.0 * radii.max())
    centres = synth._place_centres(radii, box, 0.5, rng)
    return synth.cluster(level, radii, centres)


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1905_01341_gb300 import build

    build.build()


def test_geometry_matches_oracle():
    bem = _bem()
    for mesh in (synth.workload_single_sphere()[0], small_cluster(3)):
        ctx = make_ctx(mesh, mvp=bem.BEM_MVP_DIRECT, precision=bem.BEM_PREC_FP64)
        s = np.zeros(mesh.n)
        n = np.zeros(3 * mesh.n)
        ld = np.zeros(mesh.n)
        md = np.zeros(mesh.n)
        bem.bem_get_geometry(ctx.ctx, s, n, ld, md)
        ref = oracle.BemOperator(mesh.xyz, mesh.tri)
        assert np.allclose(s, ref.s, rtol=1e-13, atol=0)
        assert np.allclose(n.reshape(3, -1).T, ref.n, rtol=0, atol=1e-13)
        assert rel(md, ref.mdiag) < 1e-11
        assert rel(ld, ref.ldiag) < 1e-11
        ctx.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-6)])
def test_direct_apply_matches_oracle(prec, tol):
    bem = _bem()
    mesh = small_cluster(3)  # 1926 vertices: 15 full tiles of 128 and a ragged one
    ctx = make_ctx(mesh, mvp=bem.BEM_MVP_DIRECT, precision=prec, diag_precision=0)
    ref = oracle.BemOperator(mesh.xyz, mesh.tri)
    rng = np.random.Generator(np.random.PCG64(3))
    xL, xM = rng.standard_normal(mesh.n), rng.standard_normal(mesh.n)
    for f, g in ((1.0, 0.0), (0.0, 1.0), (0.7, -1.3)):
        out = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
        ctx.apply(f, dev(xL), g, dev(xM), out)
        exp = ref.apply(f, xL, g, xM)
        assert rel(out.cpu().numpy(), exp) < tol, (f, g)
    ctx.close()


@pytest.mark.parametrize("prec,p,tol", [(0, 17, 1e-6), (1, 14, 1e-5)])
def test_fmm_apply_matches_oracle(prec, p, tol):
    bem = _bem()
    mesh = small_cluster(20, 3, seed=11)  # 12840 vertices
    ctx = make_ctx(mesh, mvp=bem.BEM_MVP_FMM, precision=prec, p_fmm=p, leaf_target=32)
    st = ctx.stats()
    assert st["levels"] >= 3 and st["m2l_pairs"] > 0
    ref = oracle.BemOperator(mesh.xyz, mesh.tri)
    rng = np.random.Generator(np.random.PCG64(5))
    xL, xM = rng.standard_normal(mesh.n), rng.standard_normal(mesh.n)
    for f, g in ((1.0, 0.0), (0.0, 1.0), (0.7, -1.3)):
        out = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
        ctx.apply(f, dev(xL), g, dev(xM), out)
        exp = ref.apply(f, xL, g, xM)
        assert rel(out.cpu().numpy(), exp) < tol, (f, g, rel(out.cpu().numpy(), exp))
    ctx.close()


def test_config1_solve_matches_oracle_and_closed_form():
    bem = _bem()
    mesh, phi = synth.workload_single_sphere()
    ref = oracle.BemOperator(mesh.xyz, mesh.tri)
    qref, it_ref, _, _ = oracle.solve(ref, phi, tol=1e-10)
    ctx = make_ctx(mesh, mvp=bem.BEM_MVP_DIRECT, precision=bem.BEM_PREC_FP64, gmres_tol=1e-10)
    q = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
    it, rr = ctx.solve(dev(phi), q)
    qn = q.cpu().numpy()
    assert rr <= 1e-10
    assert abs(it - it_ref) <= 1
    assert rel(qn, qref) < 1e-9
    qex = -1.0 - 0.3 * (phi - 1.0) / 0.1
    assert rel(qn, qex) < 0.01
    st = ctx.stats()
    assert st["last_mvps"] == it + 2
    ctx.close()


def test_host_pointers_match_device_pointers():
    bem = _bem()
    mesh, phi = synth.workload_single_sphere()
    ctx = bem.BemContext(mvp=bem.BEM_MVP_DIRECT, precision=bem.BEM_PREC_FP64, gmres_tol=1e-10)
    ctx.upload_mesh(mesh)  # host arrays
    ctx.build()
    out_h = np.zeros(mesh.n)
    ctx.apply(0.0, None, 1.0, phi, out_h)
    out_d = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
    ctx.apply(0.0, None, 1.0, dev(phi), out_d)
    assert np.array_equal(out_h, out_d.cpu().numpy())
    qh = np.zeros(mesh.n)
    ctx.solve(phi, qh)
    qd = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
    ctx.solve(dev(phi), qd)
    assert np.array_equal(qh, qd.cpu().numpy())
    ctx.close()


def test_error_codes():
    bem = _bem()
    mesh = synth.sphere_bubble(2)
    ctx = bem.BemContext()
    out = np.zeros(mesh.n)
    with pytest.raises(bem.BemError) as e:
        ctx.apply(1.0, np.ones(mesh.n), 0.0, None, out)
    assert e.value.code == bem.BEM_ERR_NOT_BUILT
    bad = mesh.vert_off.copy()
    bad[-1] += 1
    with pytest.raises(bem.BemError) as e:
        ctx.upload(mesh.xyz_soa(), mesh.tri_soa(), bad, mesh.tri_off)
    assert e.value.code == bem.BEM_ERR_ARG
    tri = mesh.tri_soa().copy()
    tri[0, 0] = mesh.n + 5
    with pytest.raises(bem.BemError) as e:
        ctx.upload(mesh.xyz_soa(), tri, mesh.vert_off, mesh.tri_off)
    assert e.value.code == bem.BEM_ERR_MESH
    with pytest.raises(bem.BemError) as e:
        bem.BemContext(p_fmm=40)
    assert e.value.code == bem.BEM_ERR_ARG
    ctx.close()


@pytest.fixture(scope="module")
def l6_reference():
    mesh, phi = synth.workload_single_bubble_l6()
    ref = oracle.BemOperator(mesh.xyz, mesh.tri)
    rng = np.random.Generator(np.random.PCG64(8))
    x = rng.standard_normal(mesh.n)
    return mesh, phi, ref, x, ref.apply(1.0, x, 0.0, None), ref.apply(0.0, None, 1.0, phi)


@pytest.mark.parametrize("prec", [0, 1])
def test_single_bubble_l6_p_sweep(l6_reference, prec):
    """40962-vertex perturbed sphere: FMM error against the direct oracle falls with p;
    FP64 reaches 1e-6 by p = 16, mixed precision 1e-5 by p = 14."""
    bem = _bem()
    mesh, phi, ref, x, eL, eM = l6_reference
    errs = {}
    for p in (8, 10, 12, 14, 16):
        ctx = make_ctx(mesh, mvp=bem.BEM_MVP_FMM, precision=prec, p_fmm=p)
        o1 = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
        o2 = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
        ctx.apply(1.0, dev(x), 0.0, None, o1)
        ctx.apply(0.0, None, 1.0, dev(phi), o2)
        errs[p] = max(rel(o1.cpu().numpy(), eL), rel(o2.cpu().numpy(), eM))
        ctx.close()
    print("p sweep prec=%d:" % prec, {k: "%.2e" % v for k, v in errs.items()})
    assert errs[8] > errs[12] > errs[16]
    if prec == 0:
        assert errs[16] < 1e-6
    assert errs[14] < 1e-5


def test_tensor_core_diagonal_product_single_bubble_l6(l6_reference):
    """On the 40962-vertex bubble the identities (Eqs. (s3), (s5)) magnify the far field's
    rounding enough that the 4-RHS diagonal product on the tensor cores (mode 2) about doubles
    the product error at p = 14; the automatic mode (3, the default) keeps that product on the
    CUDA cores for bubbles this fine and reproduces mode 1 exactly."""
    bem = _bem()
    mesh, phi, ref, x, eL, eM = l6_reference
    errs, outs = {}, {}
    for tc in (1, 2, 3):
        ctx = make_ctx(mesh, mvp=bem.BEM_MVP_FMM, precision=bem.BEM_PREC_MIXED, p_fmm=14, m2l_tensor_cores=tc)
        o1 = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
        o2 = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
        ctx.apply(1.0, dev(x), 0.0, None, o1)
        ctx.apply(0.0, None, 1.0, dev(phi), o2)
        outs[tc] = (o1.cpu().numpy(), o2.cpu().numpy())
        errs[tc] = (rel(outs[tc][0], eL), rel(outs[tc][1], eM))
        ctx.close()
    print("single bubble L6, p=14, mixed: (L, M) errors by m2l_tensor_cores:",
          {k: "%.2e %.2e" % v for k, v in errs.items()})
    assert all(np.array_equal(a, b) for a, b in zip(outs[3], outs[1]))
    assert max(errs[1]) < 1e-5


@pytest.mark.parametrize("prec", [0, 1])
def test_fmm_apply_is_deterministic(prec):
    """Translations are summed per target in a fixed order (no floating-point atomics), so
    repeated products are bit-identical; GMRES relies on a fixed operator."""
    bem = _bem()
    mesh = small_cluster(20, 3, seed=11)
    ctx = make_ctx(mesh, mvp=bem.BEM_MVP_FMM, precision=prec, p_fmm=10, leaf_target=32)
    x = dev(np.random.Generator(np.random.PCG64(9)).standard_normal(mesh.n))
    outs = []
    for _ in range(3):
        o = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
        ctx.apply(1.0, x, 0.5, x, o)
        outs.append(o.cpu().numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    ctx.close()


@pytest.mark.parametrize("leaf_target", [32, 128])
def test_symmetric_near_field_single_layer(leaf_target):
    """Single-layer mixed products (the GMRES products) take the symmetric near field (each pair of
    neighbour leaves evaluated once, the far leaf's shares added by a second kernel) and the
    target-major M2L: against the oracle they stay within the mixed bound, and repeated products
    are bit-identical (every share and partial is summed in a fixed order). With leaves of about
    128 points every leaf has several work units, each writing its own shares."""
    bem = _bem()
    mesh = small_cluster(20, 3, seed=11)
    ctx = make_ctx(mesh, mvp=bem.BEM_MVP_FMM, precision=bem.BEM_PREC_MIXED, p_fmm=14, leaf_target=leaf_target)
    x = np.random.Generator(np.random.PCG64(19)).standard_normal(mesh.n)
    outs = []
    for _ in range(3):
        o = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
        ctx.apply(1.0, dev(x), 0.0, None, o)
        outs.append(o.cpu().numpy())
    ctx.close()
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    ref = oracle.BemOperator(mesh.xyz, mesh.tri).apply(1.0, x, 0.0, np.zeros(mesh.n))
    err = rel(outs[0], ref)
    print("leaf target %d: single-layer product vs oracle %.2e" % (leaf_target, err))
    assert err < 1e-5


def test_residual_history_and_mvp_count():
    bem = _bem()
    mesh, phi = synth.workload_single_sphere()
    ctx = make_ctx(mesh, mvp=bem.BEM_MVP_FMM, precision=bem.BEM_PREC_FP64, p_fmm=16, gmres_tol=1e-9,
                   fixed_level=3)
    q = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
    it, rr = ctx.solve(dev(phi), q)
    h = bem.bem_get_residual_history(ctx.ctx)
    assert len(h) == it + 2  # initial residual, one estimate per iteration, final true residual
    assert h[0] == pytest.approx(1.0) and h[-1] == pytest.approx(rr) and rr <= 1e-9
    assert all(a >= b for a, b in zip(h[1:-2], h[2:-1]))  # GMRES estimates never increase
    assert ctx.stats()["last_mvps"] == it + 2
    ctx.close()


@pytest.mark.parametrize("p", [8, 14, 16])
def test_tensor_core_m2l_matches_cuda_core_m2l(p):
    """The tcgen05 M2L (three-piece BF16 split of both operands, FP32 accumulation), in both
    layouts (target-major: several classes accumulated per tile in tensor memory; pair-major:
    one row per translation), against the FP32 CUDA-core M2L: measured against the FP64 FMM at
    the same p (same truncation, so only arithmetic error is left), the tensor-core products are
    as accurate as the CUDA-core one, and stay within the mixed-precision bound of the oracle."""
    bem = _bem()
    mesh = small_cluster(20, 3, seed=11)
    rng = np.random.Generator(np.random.PCG64(12))
    xL, xM = rng.standard_normal(mesh.n), rng.standard_normal(mesh.n)
    outs = {}
    for key, prec, tc, tm in (("tc", 1, 1, 1), ("tc_pm", 1, 1, 0), ("cc", 1, 0, 1), ("f64", 0, 0, 1)):
        ctx = make_ctx(mesh, mvp=bem.BEM_MVP_FMM, precision=prec, p_fmm=p, leaf_target=32, m2l_tensor_cores=tc,
                       diag_precision=0, m2l_target_major=tm)
        o = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
        ctx.apply(0.7, dev(xL), -1.3, dev(xM), o)
        outs[key] = o.cpu().numpy()
        ctx.close()
    e_tc, e_pm, e_cc = (rel(outs[k], outs["f64"]) for k in ("tc", "tc_pm", "cc"))
    print("p=%d arithmetic error vs FP64 FMM: tensor cores %.2e (pair-major %.2e), CUDA cores %.2e"
          % (p, e_tc, e_pm, e_cc))
    assert e_tc < 2.0 * e_cc + 1e-7 and e_pm < 2.0 * e_cc + 1e-7
    if p >= 14:
        ref = oracle.BemOperator(mesh.xyz, mesh.tri).apply(0.7, xL, -1.3, xM)
        assert rel(outs["tc"], ref) < 1e-5 and rel(outs["tc_pm"], ref) < 1e-5


def test_tensor_core_diagonals_match_oracle():
    """The singular diagonals (Eqs. s3, s5) from the 4-RHS product with its M2L on the tensor
    cores (m2l_tensor_cores = 2) against the oracle's and against the same product on the CUDA
    cores: the identities cancel O(1) sums down to O(h), so they show the M2L's rounding
    magnified."""
    bem = _bem()
    mesh = small_cluster(20, 3, seed=11)
    ref = oracle.BemOperator(mesh.xyz, mesh.tri)
    errs = {}
    for tc in (2, 0):
        ctx = make_ctx(mesh, mvp=bem.BEM_MVP_FMM, precision=1, p_fmm=14, leaf_target=32, m2l_tensor_cores=tc)
        s, n, ld, md = np.zeros(mesh.n), np.zeros(3 * mesh.n), np.zeros(mesh.n), np.zeros(mesh.n)
        bem.bem_get_geometry(ctx.ctx, s, n, ld, md)
        errs[tc] = (rel(ld, ref.ldiag), rel(md, ref.mdiag))
        ctx.close()
    print("diagonals vs oracle (L, M): tensor cores %.2e %.2e, CUDA cores %.2e %.2e" % (errs[2] + errs[0]))
    for tc in (2, 0):
        assert errs[tc][0] < 1e-4 and errs[tc][1] < 1e-4
    assert errs[2][0] < 2.0 * errs[0][0] + 1e-6 and errs[2][1] < 2.0 * errs[0][1] + 1e-6


def test_mixed_tensor_core_solve_converges_below_1e6():
    """GMRES on the mixed-precision operator (tensor-core M2L) reaches 1e-7: the operator's
    rounding noise stays below the tolerance the method is run at."""
    bem = _bem()
    mesh = small_cluster(20, 3, seed=11)
    rng = np.random.Generator(np.random.PCG64(15))
    phi = synth.cluster_potential(mesh, 4, 0.1, rng) + 1.0
    ctx = make_ctx(mesh, mvp=bem.BEM_MVP_FMM, precision=bem.BEM_PREC_MIXED, p_fmm=14, leaf_target=32,
                   gmres_tol=1e-7, gmres_maxit=300, gmres_restart=100)
    q = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
    it, rr = ctx.solve(dev(phi), q, raise_on_noconv=False)
    print("mixed tensor-core solve: %d iterations, relres %.2e" % (it, rr))
    assert rr <= 1e-7
    ctx.close()


def test_jacobi_preconditioned_gmres_same_solution_fewer_iterations():
    """Right Jacobi preconditioning (optional; the paper's GMRES is unpreconditioned) solves
    the same system: both solutions agree with the oracle's to the solve tolerance, and on a
    cluster of bubbles with different radii it needs fewer iterations."""
    bem = _bem()
    mesh = small_cluster(12, 3, seed=13)
    rng = np.random.Generator(np.random.PCG64(14))
    phi = synth.cluster_potential(mesh, 4, 0.1, rng) + 1.0
    ref = oracle.BemOperator(mesh.xyz, mesh.tri)
    qref, _, _, _ = oracle.solve(ref, phi, tol=1e-12, maxit=400, restart=100)
    res = {}
    for pc in (0, 1):
        ctx = make_ctx(mesh, mvp=bem.BEM_MVP_DIRECT, precision=bem.BEM_PREC_FP64, gmres_tol=1e-10,
                       gmres_maxit=400, gmres_restart=100, gmres_precond=pc)
        q = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
        it, rr = ctx.solve(dev(phi), q)
        assert rr <= 1e-10
        res[pc] = (it, q.cpu().numpy())
        ctx.close()
    assert rel(res[0][1], qref) < 1e-8 and rel(res[1][1], qref) < 1e-8
    assert res[1][0] < res[0][0]


@pytest.mark.parametrize("prec", [0, 1])
def test_bubble_block_preconditioner_same_solution_far_fewer_iterations(prec):
    """Right bubble-block preconditioning (gmres_precond = 2: per distinct bubble shape, the
    inverse of the isolated bubble's single-layer block) solves the same system: the solution
    agrees with the oracle's to the solve tolerance, on a cluster that mixes two mesh levels
    (two shapes) and radii, with far fewer iterations than without it."""
    bem = _bem()
    rng = np.random.Generator(np.random.PCG64(31))
    parts = []
    for lev, nb in ((2, 6), (3, 5)):
        radii = np.exp(0.3 * rng.standard_normal(nb))
        centres = synth._place_centres(radii, 4.0 * nb ** (1 / 3), 0.5, rng) + (lev - 2) * 20.0
        parts.append(synth.cluster(lev, radii, centres))
    mesh, _, _ = synth.concat_meshes(parts)
    phi = synth.cluster_potential(mesh, 4, 0.1, rng) + 1.0
    ref = oracle.BemOperator(mesh.xyz, mesh.tri)
    qref, _, _, _ = oracle.solve(ref, phi, tol=1e-12, maxit=400, restart=100)
    tol = 1e-10 if prec == 0 else 1e-7
    its = {}
    for pc in (0, 2):
        ctx = make_ctx(mesh, mvp=bem.BEM_MVP_DIRECT, precision=prec, gmres_tol=tol, gmres_maxit=400,
                       gmres_restart=100, gmres_precond=pc)
        q = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
        it, rr = ctx.solve(dev(phi), q)
        assert rr <= tol
        # mixed products are accurate to 1e-5; the solve magnifies that by the conditioning,
        # bounded here by 50 as in the cluster test
        assert rel(q.cpu().numpy(), qref) < (1e-8 if prec == 0 else 5e-4), pc
        its[pc] = it
        ctx.close()
    print("iterations: none %d, bubble blocks %d" % (its[0], its[2]))
    assert its[2] * 2 < its[0]


def test_bubble_block_preconditioner_inverts_each_isolated_block():
    """bem_precond_apply (z = P y) against the oracle. The bubbles are exact scaled and
    translated copies of two icospheres (levels 2 and 3: two connectivity classes, interleaved
    in the vertex order), so bubble m's block of P is the inverse of its own isolated
    single-layer block, and the oracle's single layer of that bubble alone maps z_m back to y_m.
    The 260 level-2 bubbles span two bubble tiles of the tensor-core product (the second
    ragged), their 162 rows two ragged row tiles, the level-3 blocks six (ragged), K ragged in
    both. Mixed precision (split BF16 operands, FP32 accumulation) agrees with the FP64 product
    to FP32 accuracy and repeats bit for bit."""
    bem = _bem()
    rng = np.random.Generator(np.random.PCG64(43))
    nb = 263
    levels = np.full(nb, 2)
    levels[[0, 131, 262]] = 3
    radii = np.exp(0.3 * rng.standard_normal(nb))
    centres = synth._place_centres(radii, 4.0 * nb ** (1 / 3), 0.5, rng)
    mesh = synth.cluster(levels, radii, centres)
    y = rng.standard_normal(mesh.n)
    z = {}
    for prec in (0, 1):
        ctx = make_ctx(mesh, mvp=bem.BEM_MVP_DIRECT, precision=prec, gmres_precond=2)
        out = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
        ctx.precond_apply(dev(y), out)
        z[prec] = out.cpu().numpy()
        if prec == 1:
            again = torch.zeros_like(out)
            ctx.precond_apply(dev(y), again)
            assert torch.equal(out, again)
        ctx.close()
    print("mixed vs FP64 product: %.2e" % rel(z[1], z[0]))
    assert rel(z[1], z[0]) < 5e-6  # FP32 accumulation; a dropped cross term of the split is ~1.5e-5
    for m in (0, 1, 130, 131, 132, 257, 258, 261, 262):
        a, b = mesh.vert_off[m], mesh.vert_off[m + 1]
        op = oracle.BemOperator(mesh.xyz[a:b], mesh.tri[mesh.tri_off[m]:mesh.tri_off[m + 1]] - a)
        for prec, tol in ((0, 1e-9), (1, 3e-5)):
            back = op.apply(1.0, z[prec][a:b], 0.0, None)
            assert rel(back, y[a:b]) < tol, (m, prec, rel(back, y[a:b]))


def test_depth_autotuner_keeps_the_operator():
    """leaf_target = 0 times one product at three depths on the first build and keeps the
    fastest; the product at the chosen depth still matches the oracle, and a solve straight
    after the tuning converges as fast as at a fixed depth (the tuning's own tables are gone)."""
    bem = _bem()
    mesh = small_cluster(40, 3, seed=21)
    rng = np.random.Generator(np.random.PCG64(22))
    x = rng.standard_normal(mesh.n)
    ref = oracle.BemOperator(mesh.xyz, mesh.tri)
    recv = oracle.checkpoint_receivers(mesh.n, 2000, 3)
    e = ref.apply(1.0, x, 0.0, None, recv)
    phi = synth.cluster_potential(mesh, 4, 0.1, rng) + 1.0
    out, its = {}, {}
    for leaf in (64, 0):
        ctx = make_ctx(mesh, mvp=bem.BEM_MVP_FMM, precision=bem.BEM_PREC_MIXED, p_fmm=14, leaf_target=leaf,
                       gmres_tol=1e-6, gmres_maxit=300)
        o = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
        ctx.apply(1.0, dev(x), 0.0, None, o)
        out[leaf] = (o.cpu().numpy(), ctx.stats()["levels"])
        q = torch.zeros(mesh.n, dtype=torch.float64, device="cuda")
        its[leaf], _ = ctx.solve(dev(phi), q)
        ctx.close()
    print("levels fixed-rule %d, tuned %d; iterations %d / %d" % (out[64][1], out[0][1], its[64], its[0]))
    assert abs(out[0][1] - out[64][1]) <= 1
    assert rel(out[0][0][recv], e) < 1e-5
    assert its[0] <= its[64] + 3

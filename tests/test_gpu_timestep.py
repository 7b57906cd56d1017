"""Parity of the device time step (bem_step) with the CPU oracle's time step, and a spherical
bubble against the Rayleigh-Plesset equation (Section 4.1)."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import rp
from oracle import timestep as ts

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _bem():
    from paper_1905_01341_gb300 import bem

    return bem


def two_bubbles():
    radii = np.array([1.0, 0.8])
    centres = np.array([[0.0, 0.0, 0.0], [2.6, 0.4, -0.3]])
    mesh = synth.cluster(2, radii, centres)
    rng = np.random.Generator(np.random.PCG64(4))
    phi = synth.cluster_potential(mesh, 3, 0.05, rng) - 1.0
    return mesh, phi


@pytest.mark.parametrize("pf,order,corrector,rk", [(4, 6, 0, 4), (0, 6, 0, 4), (4, 4, 1, 5), (4, 5, 1, 6),
                                                    (4, 3, 0, 6), (4, 6, 1, 4)])
def test_time_steps_match_oracle(pf, order, corrector, rk):
    """Seven steps of a two-bubble system with each of Section 3.5's schemes: a Runge-Kutta start
    of order rk while fewer than order - 1 past right-hand sides exist, then Adams-Bashforth of
    that order (with the Adams-Moulton corrector when set). FP64 direct products and GMRES to
    1e-12 on both sides; states agree to 1e-8 relative."""
    bem = _bem()
    mesh, phi = two_bubbles()
    phys = ts.Physics(pf=pf, gmres_tol=1e-12, pa=0.8, ab_order=order, corrector=bool(corrector), rk_order=rk)
    sysm = ts.BubbleSystem(mesh.xyz, mesh.tri, mesh.vert_off, mesh.tri_off, phys)
    st = ts.State(xyz=mesh.xyz.copy(), phi=phi.copy())
    ctx = bem.BemContext(mvp=bem.BEM_MVP_DIRECT, precision=bem.BEM_PREC_FP64, gmres_tol=1e-12)
    ctx.upload_mesh(mesh)
    sp = bem.bem_step_params_default(pf=pf, pa=0.8, ab_order=order, corrector=corrector, rk_order=rk)
    bem.bem_step_init(ctx.ctx, phi, sp)
    xyz = np.zeros(3 * mesh.n)
    ph = np.zeros(mesh.n)
    stages = {4: 4, 5: 6, 6: 7}[rk]
    for k in range(7):
        st = sysm.step(st)
        info = bem.bem_step(ctx.ctx)
        t = bem.bem_step_get_state(ctx.ctx, xyz, ph)
        assert info["rhs_calls"] == (stages if k < order - 1 else 1 + corrector)
        assert t == pytest.approx(st.t, rel=1e-14)
        assert abs(info["dt"] - sysm.dt) < 1e-15
        disp_ref = st.xyz - mesh.xyz
        disp = xyz.reshape(3, -1).T - mesh.xyz
        assert np.linalg.norm(disp - disp_ref) < 1e-8 * np.linalg.norm(disp_ref) + 1e-13
        assert np.linalg.norm(ph - st.phi) < 1e-8 * np.linalg.norm(st.phi)
    ctx.close()


@pytest.mark.parametrize("pf", [4, 11])
def test_shape_filter_matches_oracle(pf):
    """bem_step_filter (Eqs. 3.22-3.25) against the oracle's filter on random fields: two bubble
    shapes (icosphere levels 3 and 2; the two level-3 bubbles are scaled copies and share one
    basis), a level-3 bubble's 642 vertices staged in three chunks of 256 (the last ragged), and
    P_f = pf^2 up to 121 coefficients (three row passes of the compensated kernel). FP64 to 1e-13;
    mixed precision (compensated FP32, measured 1.3e-14 and 4.0e-14) to 1e-12, far below what
    plain FP32 reaches. The device form, in place, repeats the host form bit for bit."""
    bem = _bem()
    radii = np.array([1.0, 0.7, 0.9])
    centres = np.array([[0.0, 0.0, 0.0], [2.6, 0.4, -0.3], [-0.4, 2.7, 0.5]])
    mesh = synth.cluster([3, 2, 3], radii, centres)
    rng = np.random.Generator(np.random.PCG64(9))
    X = rng.standard_normal((mesh.n, 4))
    sysm = ts.BubbleSystem(mesh.xyz, mesh.tri, mesh.vert_off, mesh.tri_off, ts.Physics(pf=pf))
    ref = sysm.apply_filter(X)
    x = np.ascontiguousarray(X.T).ravel()
    for prec, tol in ((bem.BEM_PREC_FP64, 1e-13), (bem.BEM_PREC_MIXED, 1e-12)):
        ctx = bem.BemContext(mvp=bem.BEM_MVP_DIRECT, precision=prec)
        ctx.upload_mesh(mesh)
        bem.bem_step_init(ctx.ctx, np.zeros(mesh.n), bem.bem_step_params_default(pf=pf, pa=0.8))
        y = np.zeros(4 * mesh.n)
        bem.bem_step_filter(ctx.ctx, x, y)
        err = np.linalg.norm(y.reshape(4, -1).T - ref) / np.linalg.norm(ref)
        print("pf %d, precision %d: filter error %.2e" % (pf, prec, err))
        assert err < tol
        d = torch.tensor(x, device="cuda")
        bem.bem_step_filter(ctx.ctx, d, d)
        assert np.array_equal(d.cpu().numpy(), y)
        ctx.close()


def test_spherical_bubble_against_rayleigh_plesset_mixed_fmm():
    """Single spherical bubble (642 vertices) under Pa = p0 at 200 kHz, through the mixed FMM
    path: the volume-equivalent radius follows Eq. (4.1) within 2% over 0.4 periods."""
    bem = _bem()
    mesh = synth.sphere_bubble(3, 1.0)
    ctx = bem.BemContext(mvp=bem.BEM_MVP_FMM, precision=bem.BEM_PREC_MIXED, p_fmm=12, gmres_tol=1e-7,
                         fixed_level=3)
    ctx.upload_mesh(mesh)
    sp = bem.bem_step_params_default(pf=6)
    bem.bem_step_init(ctx.ctx, np.zeros(mesh.n), sp)
    T = 2 * math.pi / sp.omega
    xyz = np.zeros(3 * mesh.n)
    ts_, rad = [0.0], [1.0]
    V0 = ts.bubble_volumes(mesh.xyz, mesh.tri, mesh.tri_off)[0]
    t = 0.0
    while t < 0.4 * T:
        info = bem.bem_step(ctx.ctx)
        assert info["nonconverged"] == 0
        t = bem.bem_step_get_state(ctx.ctx, xyz)
        V = ts.bubble_volumes(xyz.reshape(3, -1).T, mesh.tri, mesh.tri_off)[0]
        ts_.append(t)
        rad.append((V / V0) ** (1.0 / 3.0))
    a_rp, _ = rp.rayleigh_plesset(np.array(ts_), sp.sigma, sp.kappa, sp.pa, sp.omega)
    assert rad[-1] > 1.2
    assert np.max(np.abs(np.array(rad) - a_rp)) < 0.02 * a_rp.max()
    ctx.close()


def test_extrapolated_guess_same_states_fewer_iterations():
    """Adams-Bashforth solves that start from the quadratic extrapolation in t of the last three
    step-start solutions (guess = 2) reach the same states as solves that start from the
    previous solve's q (guess = 0, the paper's start), in fewer GMRES iterations. The tolerance
    is the benchmark's 1e-6, above the mixed path's rounding floor near 1e-7."""
    bem = _bem()
    mesh, phi = synth.workload_cluster(bubbles=30, level=3, seed=9)
    res = {}
    for g in (0, 2):
        ctx = bem.BemContext(mvp=bem.BEM_MVP_FMM, precision=bem.BEM_PREC_MIXED, p_fmm=14, gmres_tol=1e-6,
                             gmres_precond=2)
        ctx.upload_mesh(mesh)
        bem.bem_step_init(ctx.ctx, phi, bem.bem_step_params_default(pf=6, guess=g))
        iters = 0
        for k in range(10):
            info = bem.bem_step(ctx.ctx)
            assert info["nonconverged"] == 0
            if k >= 5:
                iters += info["gmres_iters"]
        xyz = np.zeros(3 * mesh.n)
        ph = np.zeros(mesh.n)
        bem.bem_step_get_state(ctx.ctx, xyz, ph)
        res[g] = (iters, xyz.reshape(3, -1).T.copy(), ph)
        ctx.close()
    print("AB6 GMRES iterations over 5 steps: guess 0 %d, guess 2 %d" % (res[0][0], res[2][0]))
    assert res[2][0] < res[0][0]
    disp = np.linalg.norm(res[0][1] - mesh.xyz)
    assert np.linalg.norm(res[2][1] - res[0][1]) < 1e-4 * disp
    assert np.linalg.norm(res[2][2] - res[0][2]) < 1e-5 * np.linalg.norm(res[0][2])


def _state(ctx, n):
    bem = _bem()
    xyz, ph, q = np.zeros(3 * n), np.zeros(n), np.zeros(n)
    t = bem.bem_step_get_state(ctx.ctx, xyz, ph, q)
    return xyz, ph, q, t


def test_checkpoint_resume_repeats_the_run_bit_for_bit():
    """A run saved after its sixth step (the first Adams-Bashforth step follows five RK4 steps)
    and resumed in a fresh context, from a host and from a device buffer, repeats the original's
    next three steps exactly: FP64 FMM at a fixed depth with Jacobi-preconditioned GMRES."""
    bem = _bem()
    mesh, phi = synth.workload_cluster(bubbles=6, level=3, seed=31)
    prm = dict(mvp=bem.BEM_MVP_FMM, precision=bem.BEM_PREC_FP64, p_fmm=10, fixed_level=3, gmres_tol=1e-9,
               gmres_precond=1)
    sp = bem.bem_step_params_default(pf=6, pa=0.5, guess=2)
    ctx = bem.BemContext(**prm)
    ctx.upload_mesh(mesh)
    bem.bem_step_init(ctx.ctx, phi, sp)
    for _ in range(6):
        bem.bem_step(ctx.ctx)
    size = bem.bem_step_save(ctx.ctx)
    host = np.zeros(size, np.uint8)
    assert bem.bem_step_save(ctx.ctx, host) == size
    devbuf = torch.from_numpy(host).cuda()
    ref = []
    for _ in range(3):
        ref.append((bem.bem_step(ctx.ctx), _state(ctx, mesh.n)))
    ctx.close()
    for buf in (host, devbuf):
        c2 = bem.BemContext(**prm)
        c2.upload_mesh(mesh)
        bem.bem_step_load(c2.ctx, buf)
        for info0, st0 in ref:
            info = bem.bem_step(c2.ctx)
            st = _state(c2, mesh.n)
            assert info["gmres_iters"] == info0["gmres_iters"] and info["steps"] == info0["steps"]
            assert st[3] == st0[3]
            for a, b in zip(st[:3], st0[:3]):
                assert np.array_equal(a, b)
        c2.close()
    # a checkpoint of another mesh size is refused
    other, _ = synth.workload_cluster(bubbles=5, level=3, seed=31)
    c3 = bem.BemContext(**prm)
    c3.upload_mesh(other)
    with pytest.raises(bem.BemError) as ei:
        bem.bem_step_load(c3.ctx, host)
    assert ei.value.code == bem.BEM_ERR_ARG
    with pytest.raises(bem.BemError):
        bem.bem_step_load(c3.ctx, host[:100])
    c3.close()


def test_dynamics_error_of_the_mixed_step_against_fp64():
    """The dynamics error of Eq. (eqErr), eps(t) = |x(t) - x_ref(t)| / max_tau |x_ref(tau) - x_ref(0)|
    over the surface-point coordinates, of the benchmark's mixed-precision step (p = 14, FP32 near
    field, BF16-split tensor-core M2L, GMRES to 1e-6) against the FP64 path at p = 16 with GMRES
    to 1e-10, over 20 steps of a 40-bubble cluster. The paper reports 5.3e-3 (single precision,
    p = 8, tolerance 1e-4) and 2.5e-4 (double, p = 12, 1e-5) at step 200; the bound here is the
    GMRES tolerance's share: 1e-3."""
    bem = _bem()
    mesh, phi = synth.workload_cluster(bubbles=40, level=3, seed=32)
    sp = bem.bem_step_params_default(pf=6, pa=0.5, guess=2)
    runs = {}
    for key, prm in (("mixed", dict(precision=bem.BEM_PREC_MIXED, p_fmm=14, gmres_tol=1e-6)),
                     ("ref", dict(precision=bem.BEM_PREC_FP64, p_fmm=16, gmres_tol=1e-10))):
        ctx = bem.BemContext(mvp=bem.BEM_MVP_FMM, gmres_precond=2, gmres_maxit=200, **prm)
        ctx.upload_mesh(mesh)
        bem.bem_step_init(ctx.ctx, phi, sp)
        xs = []
        for _ in range(20):
            info = bem.bem_step(ctx.ctx)
            assert info["nonconverged"] == 0
            xs.append(_state(ctx, mesh.n)[0])
        runs[key] = xs
        ctx.close()
    x0 = mesh.xyz_soa().reshape(-1)
    span = 0.0
    eps = []
    for x, xr in zip(runs["mixed"], runs["ref"]):
        span = max(span, np.linalg.norm(xr - x0))
        eps.append(np.linalg.norm(x - xr) / span)
    print("eps(t) over 20 steps:", ["%.2e" % e for e in eps])
    assert max(eps) < 1e-3


def test_unfiltered_mesh_destabilises_and_the_filter_keeps_it_smooth():
    """Section 4.1 reports that without the spherical filter the mesh of a bubble driven by the
    acoustic field destabilises within about 40-50 steps (52, 40 and 37 steps at N = 642, 2562,
    10245). A spherical bubble (642 vertices) under Pa = p0 at 200 kHz, stepped with p_f = 0 and
    with p_f = 6: the non-spherical part of the surface (the spread of the vertex distances from
    the centroid relative to their mean) grows without the filter until it exceeds 1 % (or the
    step fails), and stays below 0.1 % with it over the same steps."""
    bem = _bem()
    mesh = synth.sphere_bubble(3, 1.0)

    def run(pf, nsteps):
        ctx = bem.BemContext(mvp=bem.BEM_MVP_DIRECT, precision=bem.BEM_PREC_FP64, gmres_tol=1e-10)
        ctx.upload_mesh(mesh)
        bem.bem_step_init(ctx.ctx, np.zeros(mesh.n), bem.bem_step_params_default(pf=pf, pa=1.0))
        xyz = np.zeros(3 * mesh.n)
        hist = []
        for k in range(nsteps):
            try:
                bem.bem_step(ctx.ctx)
            except bem.BemError:
                hist.append(np.inf)
                break
            bem.bem_step_get_state(ctx.ctx, xyz)
            x = xyz.reshape(3, -1).T
            r = np.linalg.norm(x - x.mean(axis=0), axis=1)
            hist.append(float(np.std(r) / np.mean(r)) if np.all(np.isfinite(r)) else np.inf)
            if not np.isfinite(hist[-1]) or hist[-1] > 1e-2:
                break
        ctx.close()
        return hist

    raw = run(0, 200)
    print("unfiltered non-sphericity by step:", ["%.1e" % v for v in raw[::10]], "crossed 1%% at step %d" % len(raw))
    assert len(raw) < 200 and not raw[-1] <= 1e-2
    flt = run(6, len(raw))
    print("filtered: max %.2e over %d steps" % (max(flt), len(flt)))
    assert len(flt) == len(raw) and max(flt) < 1e-3


def test_toroidal_bubble_steps_match_oracle():
    """A ring-shaped bubble (Euler characteristic 0) takes the toroidal filter of Section 3.6
    (2D Fourier basis of the torus angles, Eq. (spherical7)); a spherical bubble beside it keeps
    the spherical one. Five RK4 steps of the pair: FP64 direct products and GMRES to 1e-12 on
    both sides, states agree to 1e-8 relative."""
    bem = _bem()
    torus = synth.torus_bubble(1.5, 0.5, 24, 12, axis=(0.2, 0.1, 1.0))
    sphere = synth.sphere_bubble(2, 0.6, centre=(0.3, 0.2, 2.4))
    mesh = synth.concat_meshes([torus, sphere])[0]
    rng = np.random.Generator(np.random.PCG64(7))
    phi = 0.05 * rng.standard_normal(mesh.n)
    phi = phi - phi.mean() - 1.0
    phys = ts.Physics(pf=6, gmres_tol=1e-12, pa=0.8)
    sysm = ts.BubbleSystem(mesh.xyz, mesh.tri, mesh.vert_off, mesh.tri_off, phys)
    assert [f[1].shape[1] for f in sysm.filters] == [49, 36]
    st = ts.State(xyz=mesh.xyz.copy(), phi=phi.copy())
    ctx = bem.BemContext(mvp=bem.BEM_MVP_DIRECT, precision=bem.BEM_PREC_FP64, gmres_tol=1e-12)
    ctx.upload_mesh(mesh)
    bem.bem_step_init(ctx.ctx, phi, bem.bem_step_params_default(pf=6, pa=0.8))
    xyz = np.zeros(3 * mesh.n)
    ph = np.zeros(mesh.n)
    for _ in range(5):
        st = sysm.step(st)
        bem.bem_step(ctx.ctx)
        bem.bem_step_get_state(ctx.ctx, xyz, ph)
        disp_ref = st.xyz - mesh.xyz
        disp = xyz.reshape(3, -1).T - mesh.xyz
        assert np.linalg.norm(disp - disp_ref) < 1e-8 * np.linalg.norm(disp_ref) + 1e-13
        assert np.linalg.norm(ph - st.phi) < 1e-8 * np.linalg.norm(st.phi)
    ctx.close()


def test_state_round_trip_through_host_memory_leaves_the_run_unchanged():
    """bem_step_set_state with the state just read by bem_step_get_state (the state held in host
    memory between steps) continues the integration exactly as without the round trip."""
    bem = _bem()
    mesh, phi = synth.workload_cluster(bubbles=4, level=3, seed=33)
    prm = dict(mvp=bem.BEM_MVP_FMM, precision=bem.BEM_PREC_FP64, p_fmm=10, fixed_level=3, gmres_tol=1e-9,
               gmres_precond=1)
    out = []
    for roundtrip in (False, True):
        ctx = bem.BemContext(**prm)
        ctx.upload_mesh(mesh)
        bem.bem_step_init(ctx.ctx, phi, bem.bem_step_params_default(pf=6, pa=0.5))
        for k in range(8):
            if roundtrip and k >= 5:
                xyz, ph, q, _ = _state(ctx, mesh.n)
                bem.bem_step_set_state(ctx.ctx, xyz, ph, q)
            bem.bem_step(ctx.ctx)
        out.append(_state(ctx, mesh.n))
        ctx.close()
    for a, b in zip(out[0][:3], out[1][:3]):
        assert np.array_equal(a, b)

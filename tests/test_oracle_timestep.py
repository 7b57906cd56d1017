"""Pins for the time-step part of the oracle (Sections 3.4-3.6, Eq. (4.1)): exact cases of
the surface functions, projector properties of the shape filter, the order of the AB6/RK4
scheme, and a spherical bubble against the Rayleigh-Plesset equation."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import rp
from oracle import timestep as ts


def _flat_patch(n=6, h=0.3):
    xs = np.arange(n) * h
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), np.zeros(n * n)], axis=1)
    tri = []
    for i in range(n - 1):
        for j in range(n - 1):
            a, b, c, d = i * n + j, (i + 1) * n + j, (i + 1) * n + j + 1, i * n + j + 1
            tri += [(a, b, c), (a, c, d)]
    return xyz, np.array(tri, np.int32)


def test_tangential_velocity_exact_for_linear_potential_on_a_plane():
    # On a flat patch (all N_k = +z) Stokes' theorem is exact for linear phi, so
    # v_t = grad phi - (grad phi . n) n at every vertex.
    xyz, tri = _flat_patch()
    na, A = ts.triangle_area_vectors(xyz, tri)
    assert np.allclose(na[:, 2], A)  # counter-clockwise seen from +z
    a = np.array([0.7, -1.3, 2.1])
    phi = xyz @ a
    s = np.zeros(len(xyz))
    for c in range(3):
        np.add.at(s, tri[:, c], A / 3.0)
    nrm = np.tile([0.0, 0.0, 1.0], (len(xyz), 1))
    vt = ts.tangential_velocity(xyz, tri, phi, s, nrm)
    assert np.allclose(vt, [0.7, -1.3, 0.0], atol=1e-13)


def test_tangential_velocity_sphere_converges():
    errs = []
    for lev in (2, 3, 4):
        m = synth.sphere_bubble(lev, 1.0)
        s, n = oracle.vertex_geometry(m.xyz, m.tri)
        phi = m.xyz[:, 2].copy()  # grad phi = z-hat
        vt = ts.tangential_velocity(m.xyz, m.tri, phi, s, n)
        ez = np.array([0.0, 0.0, 1.0])
        exp = ez - (n @ ez)[:, None] * n
        errs.append(np.max(np.linalg.norm(vt - exp, axis=1)))
    assert errs[0] > errs[1] > errs[2] and errs[2] < 5e-3


def test_curvature_exact_on_a_paraboloid():
    # Vertex at the origin with normal +z and five neighbours on z = B3 x^2 + B4 x y + B5 y^2:
    # the fit is exact and H = -B3 - B5.
    B3, B4, B5 = -0.3, 0.1, -0.2
    pts = [(0.0, 0.0)] + [(math.cos(t), math.sin(t)) for t in np.linspace(0, 2 * math.pi, 6)[:-1] + 0.2]
    xyz = np.array([(0.1 * x, 0.1 * y, B3 * (0.1 * x) ** 2 + B4 * 0.01 * x * y + B5 * (0.1 * y) ** 2) for x, y in pts])
    nrm = np.zeros_like(xyz)
    nrm[:, 2] = 1.0
    nbrs = [[1, 2, 3, 4, 5]] + [[0]] * 5
    H = ts.mean_curvature(xyz, nrm, nbrs, verts=[0])
    assert abs(H[0] - (-(B3 + B5))) < 1e-12


def test_curvature_sphere_is_inverse_radius():
    R = 2.0
    m = synth.sphere_bubble(4, R)
    s, n = oracle.vertex_geometry(m.xyz, m.tri)
    H = ts.mean_curvature(m.xyz, n, ts.vertex_neighbours(m.tri, m.n))
    assert np.max(np.abs(H * R - 1.0)) < 0.02


def test_volume_exact_and_convergent():
    v = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float) * 1.5
    f = []
    for a in (0, 1):
        for b in (2, 3):
            for c in (4, 5):
                f.append((a, b, c))
    f = np.array(f, np.int32)
    cr = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
    flip = np.einsum("ij,ij->i", cr, v[f].mean(1)) < 0
    f[flip] = f[flip][:, [0, 2, 1]]
    V = ts.bubble_volumes(v + 3.0, f, np.array([0, 8]))  # translation invariant
    assert abs(V[0] - 4.0 / 3.0 * 1.5 ** 3) < 1e-13
    errs = []
    for lev in (2, 3, 4):
        m = synth.sphere_bubble(lev, 0.8, centre=(1.0, -2.0, 0.5))
        errs.append(abs(ts.bubble_volumes(m.xyz, m.tri, m.tri_off)[0] / (4 * math.pi / 3 * 0.8 ** 3) - 1))
    assert 3.5 < errs[0] / errs[1] < 4.5 and errs[2] < 3e-3


def test_filter_is_an_orthogonal_projector_onto_low_harmonics():
    v, _ = synth.icosphere(3)
    G, Gp = ts.filter_factors(v, 6)
    # basis agrees with an independent real-harmonic implementation
    for n in range(6):
        for m in range(-n, n + 1):
            assert np.allclose(G[:, n * n + n + m], synth.real_sph_harm(n, m, v), atol=1e-12)
    F = G @ Gp
    assert np.allclose(F, F.T, atol=1e-12)
    assert np.allclose(F @ F, F, atol=1e-11)
    y = synth.real_sph_harm(4, -3, v) + 0.5 * synth.real_sph_harm(1, 1, v)
    assert np.allclose(F @ y, y, atol=1e-11)
    hi = synth.real_sph_harm(9, 2, v)
    assert np.linalg.norm(F @ hi) < 0.2 * np.linalg.norm(hi)


def test_ab6_rk4_order():
    # y' = -y + cos t: halving dt shrinks the error at t = 2 by about 2^5 or more.
    def f(t, y):
        return (-y[0] + math.cos(t),)

    def exact(t):
        return 0.5 * (math.cos(t) + math.sin(t)) + 0.5 * math.exp(-t)

    errs = []
    for nsteps in (40, 80):
        dt = 2.0 / nsteps
        y, hist, t = (np.array(1.0),), [], 0.0
        for _ in range(nsteps):
            y, hist = ts.ab6_rk4_step(f, y, t, dt, hist)
            t += dt
        errs.append(abs(float(y[0]) - exact(2.0)))
    assert errs[0] / errs[1] > 20


@pytest.mark.slow
def test_spherical_bubble_follows_rayleigh_plesset():
    # Section 4.1: a spherical bubble under p_inf = p0 - Pa sin(omega t), Pa = p0, 200 kHz,
    # a0 = 10 um; the equivalent radius follows Eq. (4.1) closely over the first half period.
    mesh = synth.sphere_bubble(2, 1.0)
    phys = ts.Physics(pf=4, gmres_tol=1e-10)
    sysm = ts.BubbleSystem(mesh.xyz, mesh.tri, mesh.vert_off, mesh.tri_off, phys)
    st = ts.State(xyz=mesh.xyz.copy(), phi=np.zeros(mesh.n))
    T = 2 * math.pi / phys.omega
    ts_, radii = [0.0], [1.0]
    while st.t < 0.4 * T:
        st = sysm.step(st)
        ts_.append(st.t)
        radii.append(sysm.equivalent_radius(st.xyz)[0] / sysm.a0[0])
    a_rp, _ = rp.rayleigh_plesset(np.array(ts_), phys.sigma / sysm.a0[0] * sysm.a0[0], phys.kappa, phys.pa,
                                  phys.omega)
    err = np.max(np.abs(np.array(radii) - a_rp))
    assert radii[-1] > 1.1  # it grew under the rarefaction
    assert err < 0.02 * np.max(a_rp)


@pytest.mark.parametrize("pf", [0, 4])
def test_dphi_dt_on_a_sphere_converges_to_the_closed_form(pf):
    # Eq. (3.15) with alpha = -1 and v = n q + v_t (v_t normal to n) reduces to
    #   dphi/dt = q^2/2 - |v_t|^2/2 - (p_g - 2 sigma H) + F(t).
    # On a sphere of radius R with phi = cos(theta) at t = 0: the exterior Dirichlet solution
    # gives q = -2 cos(theta)/R, the surface gradient gives |v_t|^2 = sin(theta)^2/R^2,
    # p_g = p_g0 = 1 + 2 sigma/a0 and F(0) = 1, so as h -> 0 (H -> 1/R, a0 -> R)
    #   dphi/dt -> 2 cos(theta)^2/R^2 - sin(theta)^2/(2 R^2).
    # A sign or factor slip in the alpha v_t . v term changes the limit by O(|v_t|^2) = O(1).
    # Both sides of the time step are band-limited (degrees 1 and 2), so the shape filter
    # (p_f = 4 keeps degrees 0..3) leaves them unchanged.
    R = 1.3
    errs = []
    for lev in (2, 3, 4, 5) if pf == 0 else (2, 3, 4):
        m = synth.sphere_bubble(lev, R)
        sysm = ts.BubbleSystem(m.xyz, m.tri, m.vert_off, m.tri_off, ts.Physics(pf=pf, gmres_tol=1e-12))
        ct = m.xyz[:, 2] / np.linalg.norm(m.xyz, axis=1)
        _, dphi, q = sysm.rhs(m.xyz, ct.copy(), 0.0, None)
        assert np.max(np.abs(q + 2.0 * ct / R)) < 0.05
        exact = (2.0 * ct ** 2 - 0.5 * (1.0 - ct ** 2)) / R ** 2
        errs.append(np.max(np.abs(dphi - exact)))
    print("dphi/dt errors over levels:", ["%.3g" % e for e in errs])
    # measured: 7.1e-2, 2.0e-2, 5.6e-3, 1.9e-3 (about O(h^1.7))
    assert all(a / b > 2.5 for a, b in zip(errs[:-1], errs[1:]))
    assert errs[-1] < (2.5e-3 if pf == 0 else 7e-3)


def _order_run(nsteps, **kw):
    # y' = -y + cos t, y(0) = 1 on [0, 2]: y = (cos t + sin t)/2 + exp(-t)/2
    def f(t, y):
        return (-y[0] + math.cos(t),)

    dt = 2.0 / nsteps
    y, hist, t = (np.array(1.0),), [], 0.0
    for _ in range(nsteps):
        y, hist = ts.multistep(f, y, t, dt, hist, **kw)
        t += dt
    return abs(float(y[0]) - (0.5 * (math.cos(2.0) + math.sin(2.0)) + 0.5 * math.exp(-2.0)))


@pytest.mark.parametrize("rk", [4, 5, 6])
def test_runge_kutta_starts_reach_their_order(rk):
    # only Runge-Kutta steps (order 7 never leaves the start phase): halving dt divides the error
    # by about 2^rk
    errs = []
    for n in (10, 20, 40):
        def f(t, y):
            return (-y[0] + math.cos(t),)
        dt = 2.0 / n
        y, t = (np.array(1.0),), 0.0
        for _ in range(n):
            y, _h = ts.multistep(f, y, t, dt, [], 6, False, rk)  # empty history: always a start step
            t += dt
        errs.append(abs(float(y[0]) - (0.5 * (math.cos(2.0) + math.sin(2.0)) + 0.5 * math.exp(-2.0))))
    rate = math.log2(errs[1] / errs[2])
    assert rk - 0.3 < rate < rk + 0.7, (rk, errs)


@pytest.mark.parametrize("order,corrector", [(1, False), (2, False), (3, False), (4, False), (5, False), (6, False),
                                             (4, True), (5, True), (6, True)])
def test_adams_schemes_reach_their_order(order, corrector):
    # the multistep phase dominates at fine dt (the RK6 start is more accurate than any of them)
    errs = [_order_run(n, order=order, corrector=corrector, rk_order=6) for n in (80, 160)]
    rate = math.log2(errs[0] / errs[1])
    assert order - 0.35 < rate < order + 0.8, (order, corrector, errs)
    if corrector:  # the corrector is more accurate than the predictor of the same order
        assert errs[1] < _order_run(160, order=order, corrector=False, rk_order=6)


def test_ab6_rk4_default_is_the_family_default():
    def f(t, y):
        return (-y[0] + math.cos(t),)
    y1, h1, y2, h2, t = (np.array(1.0),), [], (np.array(1.0),), [], 0.0
    for _ in range(12):
        y1, h1 = ts.ab6_rk4_step(f, y1, t, 0.1, h1)
        y2, h2 = ts.multistep(f, y2, t, 0.1, h2)
        t += 0.1
    assert float(y1[0]) == float(y2[0])


def test_torus_mesh_and_angles():
    R, r = 2.0, 0.6
    m = synth.torus_bubble(R, r, 32, 16, centre=(0.5, -1.0, 2.0), axis=(1.0, 1.0, 0.3))
    assert ts.euler_characteristic(m.n, m.t) == 0
    assert ts.euler_characteristic(*[x.shape[0] for x in synth.icosphere(3)]) == 2
    # outward normals: positive volume close to 2 pi^2 R r^2 (inscribed polyhedron: a little less)
    V = ts.bubble_volumes(m.xyz, m.tri, m.tri_off)[0]
    assert 0.95 < V / (2 * math.pi ** 2 * R * r * r) < 1.0
    # the recovered angles are the generating ones up to a constant shift and orientation
    phi, theta = ts.torus_angles(m.xyz)
    f = 2 * math.pi * np.repeat(np.arange(32), 16) / 32
    t = 2 * math.pi * np.tile(np.arange(16), 32) / 16
    for got, want in ((phi, f), (theta, t)):
        ok = False
        for sgn in (1, -1):
            dd = np.angle(np.exp(1j * (sgn * got - want)))
            ok = ok or np.std(np.angle(np.exp(1j * (dd - dd[0])))) < 1e-9
        assert ok


def test_toroidal_filter_is_an_orthogonal_projector_onto_low_frequencies():
    m = synth.torus_bubble(2.0, 0.7, 36, 18)
    G, Gp = ts.torus_filter_factors(m.xyz, 6)
    assert G.shape == (m.n, 49)
    F = G @ Gp
    assert np.allclose(F, F.T, atol=1e-11) and np.allclose(F @ F, F, atol=1e-11)
    phi, theta = ts.torus_angles(m.xyz)
    low = np.cos(2 * theta - phi) + 0.5 * np.sin(3 * phi) - 0.2 * np.cos(theta + 3 * phi)
    assert np.allclose(F @ low, low, atol=1e-10)
    high = np.cos(7 * theta + phi)  # outside |n|, |m| <= 3
    assert np.linalg.norm(F @ high) < 1e-8 * np.linalg.norm(high) + 1e-8
    saw = (-1.0) ** np.arange(m.n)  # the grid-scale mode the filter exists to remove
    assert np.linalg.norm(F @ saw) < 0.05 * np.linalg.norm(saw)
    # a torus bubble in a system gets the toroidal filter; spheres keep the spherical one
    mesh = synth.concat_meshes([m, synth.sphere_bubble(2, 0.5, centre=(0.0, 0.0, 3.0))])[0]
    sysm = ts.BubbleSystem(mesh.xyz, mesh.tri, mesh.vert_off, mesh.tri_off, ts.Physics(pf=6))
    assert [f[1].shape[1] for f in sysm.filters] == [49, 36]

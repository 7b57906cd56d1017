"""Pins for the CPU oracle: closed forms, exact identities, brute force and library
routines that a plausible slip in the oracle (a dropped weight, a wrong sign of the dipole
kernel, a flipped normal, a missing 1/(4 pi), per-bubble instead of global identity sums)
would fail. None of these tests touches the CUDA path."""
import math
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import rp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _regular_octahedron(scale=1.0):
    v = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    f = []
    for a in (0, 1):
        for b in (2, 3):
            for c in (4, 5):
                f.append((a, b, c))
    f = np.array(f, np.int32)
    cr = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
    flip = np.einsum("ij,ij->i", cr, v[f].mean(1)) < 0
    f[flip] = f[flip][:, [0, 2, 1]]
    return v * scale, f


# ----------------------------------------------------------------------------- inputs


def test_icosphere_counts_and_orientation():
    for lev, nv in [(0, 12), (1, 42), (2, 162), (3, 642), (4, 2562)]:
        v, f = synth.icosphere(lev)
        assert v.shape == (nv, 3) and f.shape == (20 * 4 ** lev, 3)
        assert np.allclose(np.linalg.norm(v, axis=1), 1.0)
        # closed 2-manifold: Euler characteristic 2, every edge shared by two faces
        edges = {}
        for a, b, c in f:
            for e in ((a, b), (b, c), (c, a)):
                edges[e] = edges.get(e, 0) + 1
        assert all((b, a) in edges for (a, b) in edges)  # consistent orientation
        assert nv - len(edges) // 2 + f.shape[0] == 2


def test_real_sph_harm_against_scipy():
    special = pytest.importorskip("scipy.special")
    if not hasattr(special, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    rng = np.random.Generator(np.random.PCG64(0))
    d = rng.standard_normal((50, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    th = np.arccos(d[:, 2])
    ph = np.arctan2(d[:, 1], d[:, 0])
    for l in range(0, 9):
        for m in range(-l, l + 1):
            ylm = special.sph_harm_y(l, abs(m), th, ph)
            if m == 0:
                ref = ylm.real
            elif m > 0:
                ref = math.sqrt(2) * ylm.real
            else:
                ref = math.sqrt(2) * ylm.imag
            assert np.allclose(synth.real_sph_harm(l, m, d), ref, atol=1e-12)


# ----------------------------------------------------------------------------- geometry (ns1)


def test_geometry_regular_octahedron_exact():
    # Regular octahedron of circumradius R: face area sqrt(3)/2 R^2, four faces per
    # vertex, so s_j = (4/3) sqrt(3)/2 R^2, and by symmetry n_j points along r_j.
    R = 1.7
    v, f = _regular_octahedron(R)
    s, n = oracle.vertex_geometry(v, f)
    assert np.allclose(s, 4.0 / 3.0 * math.sqrt(3) / 2 * R * R, rtol=1e-14)
    assert np.allclose(n, v / R, atol=1e-15)


def test_geometry_sphere_convergence():
    errs_area, errs_n = [], []
    R = 2.0
    for lev in (2, 3, 4, 5):
        m = synth.sphere_bubble(lev, R)
        s, n = oracle.vertex_geometry(m.xyz, m.tri)
        errs_area.append(abs(s.sum() / (4 * math.pi * R * R) - 1.0))
        rhat = m.xyz / np.linalg.norm(m.xyz, axis=1, keepdims=True)
        errs_n.append(np.max(1.0 - np.einsum("ij,ij->i", n, rhat)))
    # second order in the edge length: about 4x smaller per subdivision
    for a, b in zip(errs_area, errs_area[1:]):
        assert 3.5 < a / b < 4.5
    assert errs_area[-1] < 1e-3
    assert errs_n[-1] < 1e-5 and all(e >= 0 for e in errs_n)


# ----------------------------------------------------------------------------- operators


def _brute_force(xyz, s, n, f, xL, g, xM):
    out = []
    N = len(xyz)
    for i in range(N):
        terms = []
        for j in range(N):
            if j == i:
                continue
            d = [xyz[i][k] - xyz[j][k] for k in range(3)]
            r = math.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2)
            t = f * xL[j] / r + g * xM[j] * (n[j][0] * d[0] + n[j][1] * d[1] + n[j][2] * d[2]) / r ** 3
            terms.append(s[j] * t / (4 * math.pi))
        out.append(math.fsum(terms))
    return np.array(out)


def test_offdiag_apply_matches_brute_force_tiny():
    m = synth.perturbed_sphere(1, {(2, 0): 0.1, (3, 1): 0.05})
    s, n = oracle.vertex_geometry(m.xyz, m.tri)
    rng = np.random.Generator(np.random.PCG64(11))
    xL, xM = rng.standard_normal(m.n), rng.standard_normal(m.n)
    got = oracle.offdiag_apply(m.xyz, s, n, 0.7, xL, -1.3, xM)
    ref = _brute_force(m.xyz.tolist(), s.tolist(), n.tolist(), 0.7, xL.tolist(), -1.3, xM.tolist())
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-14)
    recv = np.array([3, 0, 41, 17], np.int64)
    assert np.allclose(oracle.offdiag_apply(m.xyz, s, n, 0.7, xL, -1.3, xM, recv), ref[recv], rtol=1e-13)


def test_dense_assembly_agrees_with_apply():
    m = synth.perturbed_sphere(2, {(2, 0): 0.05})
    s, n = oracle.vertex_geometry(m.xyz, m.tri)
    L, M = oracle.offdiag_dense(m.xyz, s, n)
    x = np.random.Generator(np.random.PCG64(1)).standard_normal(m.n)
    assert np.allclose(L @ x, oracle.offdiag_apply(m.xyz, s, n, 1.0, x, 0.0, None), rtol=1e-12, atol=1e-13)
    assert np.allclose(M @ x, oracle.offdiag_apply(m.xyz, s, n, 0.0, None, 1.0, x), rtol=1e-12, atol=1e-13)


def test_double_layer_of_constant_is_minus_half():
    # Continuous identity (Gauss, Eq. (2.11) with phi = 1, q = 0): M[1] = -1/2 on S. The
    # off-diagonal quadrature converges to it at first order; with the diagonal of Eq.
    # (s3) the discrete identity holds exactly.
    errs = []
    for lev in (2, 3, 4, 5):
        m = synth.sphere_bubble(lev, 1.5)
        s, n = oracle.vertex_geometry(m.xyz, m.tri)
        off = oracle.offdiag_apply(m.xyz, s, n, 0.0, None, 1.0, np.ones(m.n))
        errs.append(np.max(np.abs(off + 0.5)))
    for a, b in zip(errs, errs[1:]):
        assert 1.7 < a / b < 2.3
    assert errs[-1] < 0.01
    m = synth.sphere_bubble(3, 1.5)
    op = oracle.BemOperator(m.xyz, m.tri)
    assert np.allclose(op.apply_M(np.ones(m.n)), -0.5, atol=1e-13)


def test_single_layer_of_uniform_density_is_radius():
    # A sphere of radius R with unit single-layer density has potential R on its surface.
    R = 2.0
    errs = []
    for lev in (2, 3, 4, 5):
        m = synth.sphere_bubble(lev, R)
        op = oracle.BemOperator(m.xyz, m.tri)
        errs.append(np.max(np.abs(op.apply_L(np.ones(m.n)) / R - 1.0)))
    for a, b in zip(errs, errs[1:]):
        assert 3.0 < a / b < 5.0
    assert errs[-1] < 5e-4


def test_linear_identity_s5_holds():
    # Eq. (s4) projected on n_i (Eq. (s5)): n_i.(L n - M r - r/2)_i = 0 for the discrete
    # operators with the identity diagonals.
    m = synth.perturbed_sphere(3, {(2, 0): 0.1, (3, 2): 0.05})
    op = oracle.BemOperator(m.xyz, m.tri)
    acc = np.zeros(m.n)
    for c in range(3):
        acc += op.n[:, c] * (op.apply_L(op.n[:, c]) - op.apply_M(m.xyz[:, c]) - 0.5 * m.xyz[:, c])
    assert np.max(np.abs(acc)) < 1e-12


def test_far_spheres_single_and_double_layer():
    # Two spheres far apart: at the first sphere the second one's uniform single layer
    # is R^2/d (charge 4 pi R^2 seen as a point), and its double layer of a constant is 0
    # (field point outside). The identity sums of Eq. (s3)/(s5) include both bubbles.
    R, D = 1.0, 40.0
    radii = np.array([R, R])
    centres = np.array([[0.0, 0, 0], [D, 0, 0]])
    mesh = synth.cluster(3, radii, centres)
    s, n = oracle.vertex_geometry(mesh.xyz, mesh.tri)
    x = np.zeros(mesh.n)
    x[642:] = 1.0
    Lfar = oracle.offdiag_apply(mesh.xyz, s, n, 1.0, x, 0.0, None)[:642]
    dist = np.linalg.norm(mesh.xyz[:642] - centres[1], axis=1)
    assert np.allclose(Lfar, s[642:].sum() / (4 * math.pi) / dist, rtol=1e-5)
    Mfar = oracle.offdiag_apply(mesh.xyz, s, n, 0.0, None, 1.0, x)[:642]
    assert np.max(np.abs(Mfar)) < 1e-6
    # identity diagonals of the pair differ from a lone sphere's only by the tiny far terms
    op1 = oracle.BemOperator(mesh.xyz[:642], mesh.tri[:1280])
    ld, md = oracle.diagonals(mesh.xyz, s, n)
    assert np.max(np.abs(md[:642] - op1.mdiag)) < 1e-6
    assert np.max(np.abs(ld[:642] - op1.ldiag)) < 1e-3 * np.max(np.abs(op1.ldiag))


@pytest.mark.parametrize("nharm", [0, 1, 2, 3])
def test_dirichlet_sphere_closed_form(nharm):
    # Exterior Dirichlet problem on a sphere of radius R with the normal out of the
    # bubble: phi = Y_n on r = R extends as (R/r)^(n+1) Y_n, so q = -(n+1)/R Y_n.
    R = 1.3
    errs = []
    for lev in (2, 3, 4):
        m = synth.sphere_bubble(lev, R)
        op = oracle.BemOperator(m.xyz, m.tri)
        phi = synth.real_sph_harm(nharm, min(nharm, 1), m.xyz)
        q, it, rr, _ = oracle.solve(op, phi, tol=1e-11)
        assert rr < 1e-10
        qex = -(nharm + 1) / R * phi
        errs.append(np.linalg.norm(q - qex) / np.linalg.norm(qex))
    assert errs[0] > errs[1] > errs[2]
    assert errs[-1] < 0.02


def test_config1_solve_gmres_vs_lu_and_closed_form():
    mesh, phi = synth.workload_single_sphere()
    op = oracle.BemOperator(mesh.xyz, mesh.tri)
    q, it, rr, nmv = oracle.solve(op, phi, tol=1e-10)
    assert rr <= 1e-10 and nmv == it + 2
    L, M = op.dense()
    b = -0.5 * phi + M @ phi
    qlu = np.linalg.solve(L, b)
    assert np.linalg.norm(q - qlu) / np.linalg.norm(qlu) < 1e-8
    y20 = (phi - 1.0) / 0.1
    qex = -1.0 - 0.3 * y20
    assert np.linalg.norm(q - qex) / np.linalg.norm(qex) < 0.01


def test_gmres_on_random_system_and_restart():
    rng = np.random.Generator(np.random.PCG64(4))
    n = 80
    A = np.eye(n) * 4 + rng.standard_normal((n, n)) / math.sqrt(n)
    b = rng.standard_normal(n)
    xref = np.linalg.solve(A, b)
    for restart in (None, 5):
        x, it, rr, _ = oracle.gmres(lambda v: A @ v, b, np.zeros(n), tol=1e-12, maxit=400,
                                    restart=restart)
        assert rr < 1e-12
        assert np.linalg.norm(x - xref) / np.linalg.norm(xref) < 1e-10
    # exact initial guess: no iteration
    x, it, rr, nmv = oracle.gmres(lambda v: A @ v, b, xref, tol=1e-10)
    assert it == 0 and nmv == 1


# ----------------------------------------------------------------------------- Rayleigh-Plesset


def _constants():
    c = {}
    with open(os.path.join(GOLDEN, "paper_constants.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                c[k] = float(v)
    return c


def test_rp_small_oscillation_frequency():
    # Linearising Eq. (4.1) about equilibrium gives the natural frequency
    # omega0^2 = 3 kappa p_g0 - 2 sigma (dimensionless), the Minnaert frequency with
    # surface tension.
    c = _constants()
    sigma = c["sigma"] / (c["p0"] * c["a0"])
    kappa = c["kappa"]
    w0 = math.sqrt(3 * kappa * (1 + 2 * sigma) - 2 * sigma)
    T0 = 2 * math.pi / w0
    t = np.linspace(0, 3 * T0, 30001)
    a, _ = rp.rayleigh_plesset(t, sigma, kappa, 0.0, 0.0, a0=1.0 + 1e-5)
    # successive maxima of a(t) are one period apart
    x = a - 1.0
    peaks = [i for i in range(1, len(x) - 1) if x[i] > x[i - 1] and x[i] >= x[i + 1]]
    period = (t[peaks[-1]] - t[peaks[0]]) / (len(peaks) - 1)
    assert abs(period / T0 - 1.0) < 2e-4


def test_rp_energy_conserved_unforced():
    sigma, kappa = 0.073, 1.4
    t = np.linspace(0, 20.0, 2001)
    a, ad = rp.rayleigh_plesset(t, sigma, kappa, 0.0, 0.0, a0=1.3)
    e = rp.rp_energy(a, ad, sigma, kappa)
    assert np.max(np.abs(e - e[0])) / abs(e[0]) < 1e-8
    assert a.min() < 0.9  # it actually oscillates


def test_rp_forced_starts_at_rest_and_grows_under_rarefaction():
    # p_inf = p0 - Pa sin(omega t): the first half-period is a rarefaction, so the bubble
    # first grows.
    c = _constants()
    sigma = c["sigma"] / (c["p0"] * c["a0"])
    omega = 2 * math.pi * c["frequency_hz"] * c["a0"] * math.sqrt(c["rho"] / c["p0"])
    t = np.linspace(0, 0.5 * 2 * math.pi / omega, 200)
    a, ad = rp.rayleigh_plesset(t, sigma, c["kappa"], 1.0, omega)
    assert a[0] == 1.0 and ad[0] == 0.0
    assert a[-1] > 1.2

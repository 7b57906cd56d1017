"""Time step of the bubble-dynamics method (paper Sections 3.4-3.6), CPU FP64 reference.

TEST INFRASTRUCTURE: part of the CPU oracle (see oracle/__init__.py).

One right-hand-side evaluation, in the paper's order:
  1. shape filter on the inputs r and phi, per bubble (Section 3.6, Eqs. (3.22)-(3.25));
  2. vertex weights and normals (Eq. (ns1)), singular diagonals (Eqs. (s3), (s5)) and the
     Dirichlet solve L q = -phi/2 + M phi by GMRES from the previous q (Section 3.8);
  3. tangential velocity from Stokes' theorem per triangle (Eqs. (3.6)-(3.11));
  4. mean curvature from a paraboloid through five neighbours (Eqs. (parab1)-(parab2));
  5. bubble volume (divergence theorem on the flat facets; the paper gives no formula) and
     polytropic gas pressure (Eq. (2.8));
  6. dr/dt = u = v + alpha v_t with alpha = -1, i.e. u = n q (Eqs. (3.13)-(3.14)), and
     dphi/dt = (alpha v_t + v/2).v - (p_g - 2 sigma H)/rho + F(t) (Eq. (3.15)), g = 0,
     F(t) = p_inf(t)/rho with p_inf = p0 - Pa sin(omega t) (Eqs. (2.5)-(2.6));
  7. shape filter on the outputs dr/dt and dphi/dt.
Time marching: 6th-order Adams-Bashforth started by 4th-order Runge-Kutta (Section 3.5),
constant step dt = C min(edge length at t = 0) (rho/Pa)^(1/2) (Eq. (3.12)).

Units: lengths by a0, pressure by p0, time by a0 (rho/p0)^(1/2), so rho = p0 = 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import BemOperator, solve

AB6 = np.array([4277.0, -7923.0, 9982.0, -7298.0, 2877.0, -475.0]) / 1440.0  # f_n, f_{n-1}, ...

# Section 3.5 names the schemes tried: Adams-Bashforth of orders 1-6, Adams-Bashforth-Moulton
# predictor-correctors of orders 4-6, and Runge-Kutta starts of orders 4-6. Coefficients of the
# k-step Adams-Bashforth formula y_{n+1} = y_n + dt sum_j b_j f_{n-j} (newest first), from the
# integral of the interpolating polynomial through f_n .. f_{n-k+1}:
ADAMS_BASHFORTH = {
    1: np.array([1.0]),
    2: np.array([3.0, -1.0]) / 2.0,
    3: np.array([23.0, -16.0, 5.0]) / 12.0,
    4: np.array([55.0, -59.0, 37.0, -9.0]) / 24.0,
    5: np.array([1901.0, -2774.0, 2616.0, -1274.0, 251.0]) / 720.0,
    6: AB6,
}
# Adams-Moulton correctors of order k: y_{n+1} = y_n + dt sum_j m_j f_{n+1-j}, j = 0 .. k-1
# (f_{n+1} first, evaluated at the predicted state).
ADAMS_MOULTON = {
    4: np.array([9.0, 19.0, -5.0, 1.0]) / 24.0,
    5: np.array([251.0, 646.0, -264.0, 106.0, -19.0]) / 720.0,
    6: np.array([475.0, 1427.0, -798.0, 482.0, -173.0, 27.0]) / 1440.0,
}
# Runge-Kutta starts (Butcher tableaux: stage nodes c, coupling matrix a, weights b). Order 4:
# the classical method; order 5: Butcher's six-stage method; order 6: Butcher's seven-stage
# method with rational coefficients.
RUNGE_KUTTA = {
    4: (np.array([0.0, 0.5, 0.5, 1.0]),
        [[], [0.5], [0.0, 0.5], [0.0, 0.0, 1.0]],
        np.array([1.0, 2.0, 2.0, 1.0]) / 6.0),
    5: (np.array([0.0, 0.25, 0.25, 0.5, 0.75, 1.0]),
        [[], [0.25], [0.125, 0.125], [0.0, -0.5, 1.0], [3.0 / 16.0, 0.0, 0.0, 9.0 / 16.0],
         [-3.0 / 7.0, 2.0 / 7.0, 12.0 / 7.0, -12.0 / 7.0, 8.0 / 7.0]],
        np.array([7.0, 0.0, 32.0, 12.0, 32.0, 7.0]) / 90.0),
    6: (np.array([0.0, 1.0 / 3.0, 2.0 / 3.0, 1.0 / 3.0, 0.5, 0.5, 1.0]),
        [[], [1.0 / 3.0], [0.0, 2.0 / 3.0], [1.0 / 12.0, 1.0 / 3.0, -1.0 / 12.0],
         [-1.0 / 16.0, 9.0 / 8.0, -3.0 / 16.0, -3.0 / 8.0], [0.0, 9.0 / 8.0, -3.0 / 8.0, -3.0 / 4.0, 0.5],
         [9.0 / 44.0, -9.0 / 11.0, 63.0 / 44.0, 18.0 / 11.0, 0.0, -16.0 / 11.0]],
        np.array([11.0, 0.0, 81.0, 81.0, -32.0, -32.0, 11.0]) / 120.0),
}


# ----------------------------------------------------------------------------- surface functions


def triangle_area_vectors(xyz, tri):
    """N_k A_k = (r2 - r1) x (r3 - r1) / 2 per triangle, and A_k."""
    r1, r2, r3 = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    na = 0.5 * np.cross(r2 - r1, r3 - r1)
    return na, np.linalg.norm(na, axis=1)


def tangential_velocity(xyz, tri, phi, s, nrm):
    """Eqs. (3.10)-(3.11): per-triangle average of n x v from the contour integral of the
    linearly interpolated phi, area-averaged to the vertices, then v_t = (n x v)_j x n_j."""
    r1, r2, r3 = xyz[tri[:, 0]], xyz[tri[:, 1]], xyz[tri[:, 2]]
    p1, p2, p3 = phi[tri[:, 0]], phi[tri[:, 1]], phi[tri[:, 2]]
    _, A = triangle_area_vectors(xyz, tri)
    nxv_k = ((r2 - r3) * p1[:, None] + (r3 - r1) * p2[:, None] + (r1 - r2) * p3[:, None]) / (2.0 * A[:, None])
    acc = np.zeros_like(xyz)
    for c in range(3):
        np.add.at(acc, tri[:, c], nxv_k * A[:, None])
    nxv_j = acc / (3.0 * s[:, None])
    return np.cross(nxv_j, nrm)


def vertex_neighbours(tri, n):
    """Sorted neighbour lists (vertices sharing an edge) of every vertex."""
    nb = [set() for _ in range(n)]
    for a, b, c in tri:
        nb[a].update((b, c))
        nb[b].update((a, c))
        nb[c].update((a, b))
    return [sorted(x) for x in nb]


def local_frame(nv):
    """Orthonormal tangent vectors (e1, e2) completing the normal n to a right-handed frame.
    e1 is the normalised projection of the coordinate axis least aligned with n."""
    ax = np.argmin(np.abs(nv))
    a = np.zeros(3)
    a[ax] = 1.0
    e1 = a - np.dot(a, nv) * nv
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(nv, e1)
    return e1, e2


def mean_curvature(xyz, nrm, nbrs, verts=None):
    """Eqs. (parab1)-(parab2): fit z = B1 x + B2 y + B3 x^2 + B4 x y + B5 y^2 through five
    neighbours in the frame centred at r_j with z along n_j; H_j = -B3 - B5. Uses the five
    lowest-index neighbours of each vertex. `verts` restricts the vertices evaluated."""
    H = np.zeros(xyz.shape[0])
    for j in (range(xyz.shape[0]) if verts is None else verts):
        e1, e2 = local_frame(nrm[j])
        Q = np.zeros((5, 5))
        z = np.zeros(5)
        for l, k in enumerate(nbrs[j][:5]):
            d = xyz[k] - xyz[j]
            x, y, zz = np.dot(d, e1), np.dot(d, e2), np.dot(d, nrm[j])
            Q[l] = (x, y, x * x, x * y, y * y)
            z[l] = zz
        B = np.linalg.solve(Q, z)
        H[j] = -B[2] - B[4]
    return H


def bubble_volumes(xyz, tri, tri_off):
    """V_m = (1/3) sum_k A_k N_k . c_k over the triangles of bubble m (c_k: centroid)."""
    na, _ = triangle_area_vectors(xyz, tri)
    cen = (xyz[tri[:, 0]] + xyz[tri[:, 1]] + xyz[tri[:, 2]]) / 3.0
    per = np.einsum("ij,ij->i", na, cen) / 3.0
    return np.array([per[tri_off[m]:tri_off[m + 1]].sum() for m in range(len(tri_off) - 1)])


# ----------------------------------------------------------------------------- shape filter


def real_sh_basis(dirs, pf):
    """Real orthonormal spherical harmonics Y_n^m, n = 0..pf-1, m = -n..n, at unit directions
    [K, 3]; columns in the order of the multi-index j = n^2 + n + m (Eq. (spherical4))."""
    d = dirs / np.linalg.norm(dirs, axis=1, keepdims=True)
    ct = np.clip(d[:, 2], -1.0, 1.0)
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    ph = np.arctan2(d[:, 1], d[:, 0])
    K = d.shape[0]
    # normalised associated Legendre functions Pbar_n^m (orthonormal in cos theta with the
    # 1/(2 pi) azimuthal factor folded in below), by the standard stable recurrences
    Pb = np.zeros((pf, pf, K))
    Pb[0, 0] = math.sqrt(1.0 / (4.0 * math.pi))
    for m in range(1, pf):
        Pb[m, m] = -math.sqrt((2 * m + 1) / (2.0 * m)) * st * Pb[m - 1, m - 1]
    for m in range(0, pf - 1):
        Pb[m + 1, m] = math.sqrt(2 * m + 3) * ct * Pb[m, m]
    for m in range(0, pf):
        for n in range(m + 2, pf):
            a = math.sqrt((4.0 * n * n - 1.0) / (n * n - m * m))
            b = math.sqrt(((n - 1.0) ** 2 - m * m) / (4.0 * (n - 1.0) ** 2 - 1.0))
            Pb[n, m] = a * (ct * Pb[n - 1, m] - b * Pb[n - 2, m])
    G = np.zeros((K, pf * pf))
    for n in range(pf):
        for m in range(-n, n + 1):
            j = n * n + n + m
            if m == 0:
                G[:, j] = Pb[n, 0]
            elif m > 0:
                G[:, j] = math.sqrt(2.0) * Pb[n, m] * np.cos(m * ph)
            else:
                G[:, j] = math.sqrt(2.0) * Pb[n, -m] * np.sin(-m * ph)
    return G


def filter_factors(dirs, pf):
    """Eqs. (3.22)-(3.25): G (N_d x P_f) and its least-squares pseudo-inverse
    G^(-1) = (G^T G)^(-1) G^T (P_f x N_d); the filter is F = G G^(-1)."""
    G = real_sh_basis(dirs, pf)
    Gp = np.linalg.solve(G.T @ G, G.T)
    return G, Gp


def euler_characteristic(n_vertices, n_triangles):
    """V - E + F of a closed triangulated surface (E = 3F/2): 2 for a sphere, 0 for a torus."""
    return n_vertices - n_triangles // 2


def torus_angles(xyz):
    """Toroidal and poloidal angles (phi, theta) of the points of a ring-shaped surface: the axis
    is the principal direction of least spread about the centroid, phi the angle about it and
    theta the angle about the centre circle (radius: the mean distance from the axis)."""
    d = xyz - xyz.mean(axis=0)
    w, v = np.linalg.eigh(d.T @ d)
    a = v[:, 0]  # smallest second moment: the axis of the ring
    e1 = v[:, 2]
    e2 = np.cross(a, e1)
    u, vv, z = d @ e1, d @ e2, d @ a
    phi = np.arctan2(vv, u)
    rho = np.hypot(u, vv)
    theta = np.arctan2(z, rho - rho.mean())
    return phi, theta


def real_torus_basis(phi, theta, pf):
    """The toroidal filter's basis (the 2D Fourier basis e^{i(n theta + m phi)}, |n|, |m| <= p_f/2,
    in its real form, Eq. (spherical7)): 1, and cos/sin(n theta + m phi) for each pair +-(n, m)
    with n > 0, or n = 0 and m > 0: (2h + 1)^2 columns, h = floor(p_f / 2)."""
    h = pf // 2
    cols = [np.ones_like(phi)]
    for n in range(0, h + 1):
        for m in range(-h, h + 1):
            if n == 0 and m <= 0:
                continue
            arg = n * theta + m * phi
            cols += [np.cos(arg), np.sin(arg)]
    return np.stack(cols, axis=1)


def torus_filter_factors(xyz, pf):
    """The toroidal filter (Section 3.6, Eq. (spherical7)): G of real_torus_basis at the points'
    torus angles and G^(-1) = (G^T G)^(-1) G^T."""
    phi, theta = torus_angles(xyz)
    G = real_torus_basis(phi, theta, pf)
    Gp = np.linalg.solve(G.T @ G, G.T)
    return G, Gp


# ----------------------------------------------------------------------------- state and RHS


@dataclass
class Physics:
    sigma: float = 0.073       # sigma / (p0 a0)
    kappa: float = 1.4
    pa: float = 1.0            # Pa / p0
    omega: float = 1.2566370614359172  # omega a0 (rho/p0)^(1/2): 200 kHz, a0 = 10 um
    courant: float = 0.1       # C of Eq. (3.12)
    pf: int = 6                # filter bandwidth p_f
    gmres_tol: float = 1e-10
    ab_order: int = 6          # Adams-Bashforth order k (1..6) after the Runge-Kutta start
    corrector: bool = False    # Adams-Moulton corrector of order k (k = 4..6): two RHS per step
    rk_order: int = 4          # Runge-Kutta order of the start steps (4, 5 or 6)


@dataclass
class State:
    xyz: np.ndarray
    phi: np.ndarray
    t: float = 0.0
    q: np.ndarray | None = None
    history: list = field(default_factory=list)  # RHS values f_n, f_{n-1}, ... (newest first)
    steps: int = 0


class BubbleSystem:
    """Fixed topology and initial data of a cluster: triangles, offsets, filters, V_m0."""

    def __init__(self, xyz0, tri, vert_off, tri_off, phys: Physics):
        self.tri = np.ascontiguousarray(tri, np.int32)
        self.vert_off = np.asarray(vert_off, np.int64)
        self.tri_off = np.asarray(tri_off, np.int64)
        self.phys = phys
        self.M = len(self.vert_off) - 1
        # one filter per distinct initial shape: bubbles whose vertex directions from the
        # centroid coincide share G and G^(-1) (the radius does not matter)
        self.filters = []
        self.filter_of = np.zeros(self.M, np.int64)
        for m in range(self.M if phys.pf > 0 else 0):
            a, b = self.vert_off[m], self.vert_off[m + 1]
            d = xyz0[a:b] - xyz0[a:b].mean(axis=0)
            d = d / np.linalg.norm(d, axis=1, keepdims=True)
            for fi, (dd, _, _) in enumerate(self.filters):
                if dd.shape == d.shape and np.allclose(dd, d, atol=1e-9):
                    self.filter_of[m] = fi
                    break
            else:
                # sphere-like bubbles (Euler characteristic 2) take the spherical filter, ring-like
                # ones (0) the toroidal filter of Eq. (spherical7)
                chi = euler_characteristic(b - a, self.tri_off[m + 1] - self.tri_off[m])
                if chi == 2:
                    G, Gp = filter_factors(d, phys.pf)
                elif chi == 0:
                    G, Gp = torus_filter_factors(xyz0[a:b], phys.pf)
                else:
                    raise ValueError("bubble %d: no shape filter for Euler characteristic %d" % (m, chi))
                self.filters.append((d, G, Gp))
                self.filter_of[m] = len(self.filters) - 1
        self.V0 = bubble_volumes(xyz0, self.tri, self.tri_off)
        self.a0 = (3.0 * self.V0 / (4.0 * math.pi)) ** (1.0 / 3.0)
        self.nbrs = vertex_neighbours(self.tri, xyz0.shape[0])
        e = np.concatenate([np.linalg.norm(xyz0[self.tri[:, a]] - xyz0[self.tri[:, b]], axis=1)
                            for a, b in ((0, 1), (1, 2), (2, 0))])
        self.dt = phys.courant * e.min() * math.sqrt(1.0 / phys.pa)

    def apply_filter(self, X):
        """x_hat = G (G^(-1) x) per bubble, for X of shape [N] or [N, k] (identity when the
        bandwidth p_f is 0)."""
        if self.phys.pf == 0:
            return X.copy()
        Y = np.empty_like(X)
        for m in range(self.M):
            a, b = self.vert_off[m], self.vert_off[m + 1]
            _, G, Gp = self.filters[self.filter_of[m]]
            Y[a:b] = G @ (Gp @ X[a:b])
        return Y

    def rhs(self, xyz, phi, t, q0):
        """Filtered (dr/dt, dphi/dt) and the new q at state (xyz, phi, t)."""
        ph = self.phys
        xf = self.apply_filter(xyz)
        pf = self.apply_filter(phi)
        op = BemOperator(xf, self.tri)
        q, _, _, _ = solve(op, pf, q0, tol=ph.gmres_tol)
        vt = tangential_velocity(xf, self.tri, pf, op.s, op.n)
        H = mean_curvature(xf, op.n, self.nbrs)
        V = bubble_volumes(xf, self.tri, self.tri_off)
        pg0 = 1.0 + 2.0 * ph.sigma / self.a0
        pg = pg0 * (self.V0 / V) ** ph.kappa
        pg_v = np.repeat(pg, np.diff(self.vert_off))
        v = op.n * q[:, None] + vt
        alpha = -1.0
        dphi = np.einsum("ij,ij->i", alpha * vt + 0.5 * v, v) - (pg_v - 2.0 * ph.sigma * H) \
            + (1.0 - ph.pa * math.sin(ph.omega * t))
        dr = v + alpha * vt  # = n q
        return self.apply_filter(dr), self.apply_filter(dphi), q

    def step(self, st: State) -> State:
        """One constant-dt step of dr/dt, dphi/dt (see ab6_rk4_step)."""
        box = {"q": st.q}

        def f(t, y):
            dr, dp, q = self.rhs(y[0], y[1], t, box["q"])
            box["q"] = q
            return (dr, dp)

        ph = self.phys
        y, hist = multistep(f, (st.xyz, st.phi), st.t, self.dt, st.history, ph.ab_order, ph.corrector, ph.rk_order)
        return State(xyz=y[0], phi=y[1], t=st.t + self.dt, q=box["q"], history=hist, steps=st.steps + 1)

    def equivalent_radius(self, xyz):
        return (3.0 * bubble_volumes(xyz, self.tri, self.tri_off) / (4.0 * math.pi)) ** (1.0 / 3.0)


def multistep(f, y, t, dt, history, order=6, corrector=False, rk_order=4):
    """One step of Section 3.5's family for y' = f(t, y), y a tuple of arrays.

    history holds f at the previous step starts, newest first. While it has fewer than order - 1
    entries the step is Runge-Kutta of rk_order (tableau RUNGE_KUTTA); afterwards Adams-Bashforth
    of `order`, y* = y_n + dt sum_j b_j f_{n-j}; with `corrector`, y_{n+1} = y_n + dt (m_0 f(t+dt, y*)
    + sum_{j>=1} m_j f_{n+1-j}) (Adams-Moulton of the same order, PECE). Returns (y_{n+1}, history
    including f_n, at most 5 entries)."""
    need = order - 1
    if len(history) < need:
        c, a, b = RUNGE_KUTTA[rk_order]
        ks = []
        for i in range(len(c)):
            yi = y
            for j, aij in enumerate(a[i]):
                if aij != 0.0:
                    yi = tuple(u + dt * aij * k for u, k in zip(yi, ks[j]))
            ks.append(f(t + c[i] * dt, yi))
        ynew = tuple(u + dt * sum(bi * k[m] for bi, k in zip(b, ks) if bi != 0.0) for m, u in enumerate(y))
        return ynew, ([ks[0]] + list(history))[:5]
    fn = f(t, y)
    hist = [fn] + list(history[:5])
    bb = ADAMS_BASHFORTH[order]
    ynew = tuple(yi + dt * sum(cj * h[i] for cj, h in zip(bb, hist)) for i, yi in enumerate(y))
    if corrector:
        mm = ADAMS_MOULTON[order]
        fp = f(t + dt, ynew)
        terms = [fp] + hist[:order - 1]
        ynew = tuple(yi + dt * sum(cj * h[i] for cj, h in zip(mm, terms)) for i, yi in enumerate(y))
    return ynew, hist[:5]


def ab6_rk4_step(f, y, t, dt, history):
    """One step of Section 3.5's scheme for y' = f(t, y), y a tuple of arrays.

    history holds f at the previous step starts, newest first. While it has fewer than 5
    entries the step is classical 4th-order Runge-Kutta; afterwards 6th-order Adams-Bashforth
    y_{n+1} = y_n + dt sum_k b_k f_{n-k}, b = (4277, -7923, 9982, -7298, 2877, -475)/1440.
    Returns (y_{n+1}, history including f_n, at most 5 entries)."""
    def axpy(a, x, yy):
        return tuple(yi + a * xi for xi, yi in zip(x, yy))

    if len(history) < 5:
        k1 = f(t, y)
        k2 = f(t + 0.5 * dt, axpy(0.5 * dt, k1, y))
        k3 = f(t + 0.5 * dt, axpy(0.5 * dt, k2, y))
        k4 = f(t + dt, axpy(dt, k3, y))
        ynew = tuple(yi + dt / 6.0 * (a + 2 * b + 2 * c + d) for yi, a, b, c, d in zip(y, k1, k2, k3, k4))
        return ynew, ([k1] + list(history))[:5]
    fn = f(t, y)
    hist = [fn] + list(history[:5])
    ynew = tuple(yi + dt * sum(c * h[i] for c, h in zip(AB6, hist)) for i, yi in enumerate(y))
    return ynew, hist[:5]

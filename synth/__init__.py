"""Seeded synthetic inputs for the bubble-cluster boundary-element workloads.

This module is shared by the CPU oracle's tests and by the CUDA path's tests and
benchmark. It only builds inputs: triangulated spheres (icospheres), bubble-cluster
placements, and smooth random surface potentials. It holds none of the method's
arithmetic (no vertex weights, normals, Green's-function sums, diagonal identities,
solves or time stepping), so both sides can use it without sharing method code.

Workload shapes follow the paper's examples: icosphere meshes of 642 vertices per bubble
(Section 4), clusters of many such bubbles with centre spacing about four radii
(Section 4.3), and random uniform points in a cube for the FMM accuracy study (Table 1).

Every generator takes an explicit seed and uses numpy's PCG64, so each input is
reproducible across machines.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Mesh",
    "icosphere",
    "real_sph_harm",
    "sphere_bubble",
    "perturbed_sphere",
    "cluster",
    "random_cube_points",
    "workload_single_sphere",
    "workload_single_bubble_l6",
    "workload_cluster",
    "workload_uneven_clusters",
    "concat_meshes",
]


@dataclass
class Mesh:
    """A multi-bubble triangular surface mesh.

    xyz:      float64 [N, 3] vertex coordinates (the collocation points).
    tri:      int32 [T, 3] global vertex indices, counter-clockwise when seen from the
              liquid, so the right-hand normal points out of the bubble.
    vert_off: int64 [M+1] bubble m owns vertices vert_off[m]:vert_off[m+1].
    tri_off:  int64 [M+1] bubble m owns triangles tri_off[m]:tri_off[m+1].
    centres, radii: float64 [M, 3], [M] nominal bubble centres and radii.
    meta:     free-form description of how the mesh was made.
    """

    xyz: np.ndarray
    tri: np.ndarray
    vert_off: np.ndarray
    tri_off: np.ndarray
    centres: np.ndarray
    radii: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def t(self) -> int:
        return int(self.tri.shape[0])

    @property
    def m(self) -> int:
        return int(self.vert_off.shape[0] - 1)

    def xyz_soa(self) -> np.ndarray:
        """Coordinates as a contiguous [3, N] array (x row, y row, z row)."""
        return np.ascontiguousarray(self.xyz.T)

    def tri_soa(self) -> np.ndarray:
        """Triangle corners as a contiguous int32 [3, T] array."""
        return np.ascontiguousarray(self.tri.T.astype(np.int32))


# --------------------------------------------------------------------------------------
# icosphere
# --------------------------------------------------------------------------------------

_ICO_CACHE: dict[int, tuple[np.ndarray, np.ndarray]] = {}


def _ico_base() -> tuple[np.ndarray, list[tuple[int, int, int]]]:
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array(
        [
            [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
            [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
            [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1],
        ],
        dtype=np.float64,
    )
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = [
        (0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
        (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
        (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
        (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1),
    ]
    return v, f


def icosphere(level: int) -> tuple[np.ndarray, np.ndarray]:
    """Unit icosphere after `level` 4-to-1 subdivisions.

    Returns (xyz float64 [10*4^level+2, 3], tri int32 [20*4^level, 3]). Level 2, 3, 4 and 6
    give 162, 642, 2562 and 40962 vertices. Triangles are counter-clockwise seen from
    outside. The result is deterministic and cached.
    """
    if level < 0:
        raise ValueError("level must be >= 0")
    if level in _ICO_CACHE:
        v, f = _ICO_CACHE[level]
        return v.copy(), f.copy()
    verts, faces = _ico_base()
    vlist = [row for row in verts]
    for _ in range(level):
        cache: dict[tuple[int, int], int] = {}

        def mid(a: int, b: int) -> int:
            key = (a, b) if a < b else (b, a)
            idx = cache.get(key)
            if idx is None:
                p = vlist[a] + vlist[b]
                p = p / np.linalg.norm(p)
                idx = len(vlist)
                vlist.append(p)
                cache[key] = idx
            return idx

        nf = []
        for (a, b, c) in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    v = np.array(vlist, dtype=np.float64)
    f = np.array(faces, dtype=np.int32)
    # Orient every face counter-clockwise seen from outside (outward right-hand normal).
    cr = np.cross(v[f[:, 1]] - v[f[:, 0]], v[f[:, 2]] - v[f[:, 0]])
    flip = np.einsum("ij,ij->i", cr, v[f].mean(axis=1)) < 0
    f[flip] = f[flip][:, [0, 2, 1]]
    _ICO_CACHE[level] = (v, f)
    return v.copy(), f.copy()


# --------------------------------------------------------------------------------------
# real spherical harmonics used to build inputs (orthonormal on the unit sphere,
# Condon-Shortley phase)
# --------------------------------------------------------------------------------------


def real_sph_harm(l: int, m: int, dirs: np.ndarray) -> np.ndarray:
    """Real orthonormal spherical harmonic Y_l^m evaluated at unit directions [K, 3].

    m > 0 uses cos(m phi), m < 0 uses sin(|m| phi); the integral of Y^2 over the unit
    sphere is 1. Used only to synthesise surface shapes and potentials.
    """
    d = np.asarray(dirs, dtype=np.float64)
    r = np.linalg.norm(d, axis=1)
    ct = np.clip(d[:, 2] / r, -1.0, 1.0)
    st = np.sqrt(np.maximum(0.0, 1.0 - ct * ct))
    ph = np.arctan2(d[:, 1], d[:, 0])
    am = abs(m)
    # associated Legendre P_l^am(ct) with Condon-Shortley phase, via the standard
    # three-term recurrence in l starting from P_am^am.
    pmm = np.ones_like(ct)
    fact = 1.0
    for _ in range(am):
        pmm = -pmm * fact * st
        fact += 2.0
    if l == am:
        plm = pmm
    else:
        pmm1 = ct * (2 * am + 1) * pmm
        if l == am + 1:
            plm = pmm1
        else:
            pll = pmm1
            for ll in range(am + 2, l + 1):
                pll = ((2 * ll - 1) * ct * pmm1 - (ll + am - 1) * pmm) / (ll - am)
                pmm, pmm1 = pmm1, pll
            plm = pll
    norm = math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - am) / math.factorial(l + am))
    if m == 0:
        return norm * plm
    if m > 0:
        return math.sqrt(2.0) * norm * plm * np.cos(am * ph)
    return math.sqrt(2.0) * norm * plm * np.sin(am * ph)


def _sh_series(coef: dict[tuple[int, int], float], dirs: np.ndarray) -> np.ndarray:
    out = np.zeros(dirs.shape[0])
    for (l, m), c in coef.items():
        out += c * real_sph_harm(l, m, dirs)
    return out


def random_sh_coeffs(lmax: int, rng: np.random.Generator, scale: float = 1.0) -> dict:
    """N(0, scale^2) coefficients for every (l, m) with l <= lmax, in (l, m) order."""
    return {(l, m): scale * rng.standard_normal() for l in range(lmax + 1) for m in range(-l, l + 1)}


# --------------------------------------------------------------------------------------
# single bubbles
# --------------------------------------------------------------------------------------


def _single(xyz: np.ndarray, tri: np.ndarray, centre, radius, meta) -> Mesh:
    return Mesh(
        xyz=np.ascontiguousarray(xyz, dtype=np.float64),
        tri=np.ascontiguousarray(tri, dtype=np.int32),
        vert_off=np.array([0, xyz.shape[0]], dtype=np.int64),
        tri_off=np.array([0, tri.shape[0]], dtype=np.int64),
        centres=np.asarray([centre], dtype=np.float64),
        radii=np.asarray([radius], dtype=np.float64),
        meta=meta,
    )


def sphere_bubble(level: int, radius: float = 1.0, centre=(0.0, 0.0, 0.0)) -> Mesh:
    """One spherical bubble: icosphere of the given level scaled and shifted."""
    v, f = icosphere(level)
    c = np.asarray(centre, dtype=np.float64)
    return _single(v * radius + c, f, c, radius, {"kind": "sphere", "level": level, "radius": radius})


def perturbed_sphere(level: int, shape: dict[tuple[int, int], float]) -> Mesh:
    """Icosphere whose vertices are moved radially to r = 1 + sum c_lm Y_l^m(direction)."""
    v, f = icosphere(level)
    rad = 1.0 + _sh_series(shape, v)
    return _single(v * rad[:, None], f, (0.0, 0.0, 0.0), 1.0,
                   {"kind": "perturbed_sphere", "level": level, "shape": {f"{k}": c for k, c in shape.items()}})


def torus_bubble(R: float, r: float, n_phi: int, n_theta: int, centre=(0.0, 0.0, 0.0), axis=(0.0, 0.0, 1.0)) -> Mesh:
    """A toroidal bubble: the surface ((R + r cos t) cos f, (R + r cos t) sin f, r sin t) about
    `axis` through `centre`, sampled on an n_phi x n_theta grid of the toroidal angle f and the
    poloidal angle t, each grid cell split into two triangles, counter-clockwise seen from the
    liquid (outward normals)."""
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    e1 = np.cross(a, [1.0, 0.0, 0.0] if abs(a[0]) < 0.9 else [0.0, 1.0, 0.0])
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(a, e1)
    f = 2.0 * math.pi * np.arange(n_phi) / n_phi
    t = 2.0 * math.pi * np.arange(n_theta) / n_theta
    F, T = np.meshgrid(f, t, indexing="ij")
    rho = R + r * np.cos(T)
    pts = (rho * np.cos(F))[..., None] * e1 + (rho * np.sin(F))[..., None] * e2 + (r * np.sin(T))[..., None] * a
    xyz = pts.reshape(-1, 3) + np.asarray(centre, dtype=np.float64)
    idx = lambda i, j: (i % n_phi) * n_theta + (j % n_theta)  # noqa: E731
    tri = []
    for i in range(n_phi):
        for j in range(n_theta):
            p00, p10, p11, p01 = idx(i, j), idx(i + 1, j), idx(i + 1, j + 1), idx(i, j + 1)
            tri += [(p00, p10, p11), (p00, p11, p01)]
    tri = np.array(tri, dtype=np.int32)
    # orient outward: the normal of the first triangle must point away from the tube's centre line
    c0 = np.asarray(centre, dtype=np.float64)
    v0, v1, v2 = xyz[tri[0, 0]], xyz[tri[0, 1]], xyz[tri[0, 2]]
    nrm = np.cross(v1 - v0, v2 - v0)
    mid = (v0 + v1 + v2) / 3.0 - c0
    ring = mid - np.dot(mid, a) * a
    ring = R * ring / np.linalg.norm(ring)
    if np.dot(nrm, mid - ring) < 0.0:
        tri = tri[:, [0, 2, 1]]
    return _single(xyz, tri, c0, r, {"kind": "torus", "R": R, "r": r, "n_phi": n_phi, "n_theta": n_theta})


# --------------------------------------------------------------------------------------
# clusters
# --------------------------------------------------------------------------------------


def _place_centres(radii: np.ndarray, box: float, gap: float, rng: np.random.Generator,
                   max_tries: int = 20000) -> np.ndarray:
    """Rejection-sample centres uniform in [-box/2, box/2]^3 such that every pair obeys
    |c_i - c_j| >= R_i + R_j + gap * max(R_i, R_j). A uniform grid of cell size
    (2 max R + gap max R) keeps each test local."""
    m = radii.shape[0]
    order = np.argsort(-radii, kind="stable")  # largest first: small ones fill the gaps
    rmax = float(radii.max())
    cell = 2.0 * rmax + gap * rmax
    ncell = max(1, int(box // cell))
    grid: dict[tuple[int, int, int], list[int]] = {}
    centres = np.zeros((m, 3))
    for i in order:
        for _ in range(max_tries):
            c = (rng.random(3) - 0.5) * box
            key = tuple(np.minimum(((c + box / 2) / cell).astype(int), ncell - 1))
            ok = True
            for dx in (-1, 0, 1):
                for dy in (-1, 0, 1):
                    for dz in (-1, 0, 1):
                        for j in grid.get((key[0] + dx, key[1] + dy, key[2] + dz), ()):
                            need = radii[i] + radii[j] + gap * max(radii[i], radii[j])
                            if np.sum((centres[j] - c) ** 2) < need * need:
                                ok = False
                                break
                        if not ok:
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if ok:
                centres[i] = c
                grid.setdefault(key, []).append(i)
                break
        else:
            raise RuntimeError("could not place bubble %d; enlarge the box" % i)
    return centres


def cluster(levels, radii: np.ndarray, centres: np.ndarray) -> Mesh:
    """Concatenate scaled icospheres into one mesh (bubble-major vertex order)."""
    levels = np.broadcast_to(np.asarray(levels), radii.shape)
    xs, ts, voff, toff = [], [], [0], [0]
    for lev, r, c in zip(levels, radii, centres):
        v, f = icosphere(int(lev))
        xs.append(v * r + c)
        ts.append(f + voff[-1])
        voff.append(voff[-1] + v.shape[0])
        toff.append(toff[-1] + f.shape[0])
    return Mesh(
        xyz=np.ascontiguousarray(np.concatenate(xs), dtype=np.float64),
        tri=np.ascontiguousarray(np.concatenate(ts), dtype=np.int32),
        vert_off=np.asarray(voff, dtype=np.int64),
        tri_off=np.asarray(toff, dtype=np.int64),
        centres=np.asarray(centres, dtype=np.float64),
        radii=np.asarray(radii, dtype=np.float64),
        meta={"kind": "cluster", "bubbles": int(radii.shape[0])},
    )


def cluster_potential(mesh: Mesh, lmax: int, scale: float, rng: np.random.Generator,
                      radius_scaled: bool = False) -> np.ndarray:
    """Per-bubble smooth random potential: sum over l <= lmax of N(0,1)*scale * Y_l^m of
    the direction from the bubble centre. Coefficients are drawn bubble by bubble in
    (l, m) order. With radius_scaled the series of bubble b is multiplied by its radius, so
    every bubble starts with the same velocity scale (|grad phi| ~ scale) whatever its size."""
    lm = [(l, m) for l in range(lmax + 1) for m in range(-l, l + 1)]
    coef = scale * rng.standard_normal((mesh.m, len(lm)))
    if radius_scaled:
        coef *= np.asarray(mesh.radii, dtype=np.float64)[:, None]
    phi = np.empty(mesh.n)
    basis_cache: dict[int, np.ndarray] = {}
    for b in range(mesh.m):
        a, e = int(mesh.vert_off[b]), int(mesh.vert_off[b + 1])
        d = mesh.xyz[a:e] - mesh.centres[b]
        key = e - a
        basis = basis_cache.get(key)
        # bubbles with the same vertex count are scaled copies of one icosphere, so the
        # directions (and the basis) coincide; recompute for anything else.
        if basis is None or not np.allclose(d / np.linalg.norm(d, axis=1, keepdims=True),
                                            basis_cache[(key, "dirs")], atol=1e-12):
            dirs = d / np.linalg.norm(d, axis=1, keepdims=True)
            basis = np.stack([real_sph_harm(l, m, dirs) for (l, m) in lm], axis=1)
            basis_cache[key] = basis
            basis_cache[(key, "dirs")] = dirs
        phi[a:e] = basis @ coef[b]
    return phi


def random_cube_points(n: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """n points uniform in the unit cube and N(0,1) monopole strengths (Table 1 workload)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.random((n, 3)), rng.standard_normal(n)


# --------------------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------------------


def workload_single_sphere() -> tuple[Mesh, np.ndarray]:
    """R = 1 icosphere level 3 (642 vertices, 1280 triangles); phi = 1 + 0.1 Y_2^0."""
    mesh = sphere_bubble(3, 1.0)
    phi = 1.0 + 0.1 * real_sph_harm(2, 0, mesh.xyz)
    return mesh, phi


def workload_single_bubble_l6(seed: int = 2, level: int = 6) -> tuple[Mesh, np.ndarray]:
    """Icosphere level 6 (40962 vertices) mapped radially to r = 1 + 0.05 Y_2^0 + 0.02 Y_4^0;
    phi = sum_{l<=8} c_lm Y_l^m with c_lm ~ N(0,1) (PCG64 seed)."""
    mesh = perturbed_sphere(level, {(2, 0): 0.05, (4, 0): 0.02})
    rng = np.random.Generator(np.random.PCG64(seed))
    phi = _sh_series(random_sh_coeffs(8, rng), mesh.xyz)
    return mesh, phi


def workload_cluster(bubbles: int = 5000, level: int = 3, seed: int = 3, sigma: float = 0.3,
                     gap: float = 0.5, spacing: float = 4.0, phi_lmax: int = 6,
                     phi_scale: float = 0.01, phi_radius_scaled: bool = True) -> tuple[Mesh, np.ndarray]:
    """Random polydisperse cluster: radii lognormal(0, sigma) (median 1), centres uniform in
    a cube of side L = spacing * M^(1/3) (mean centre spacing about `spacing` median radii, as
    in the paper's d = 4 a0 clusters) with pairwise gap |c_i - c_j| >= R_i + R_j +
    gap * max(R_i, R_j); every bubble an icosphere of `level`; phi per bubble a random
    SH series with l <= phi_lmax and N(0,1)*phi_scale coefficients, times the bubble's
    radius (phi_radius_scaled: the same initial velocity scale on every bubble). The series
    is an impulsive start: surfaces move at ~|phi|(l+1)/R from t = 0 until surface tension
    turns them back a quarter capillary period later, so the amplitude sets how far a bubble
    deforms; 0.01 keeps it to a few percent of the radius over a 20-step run."""
    rng = np.random.Generator(np.random.PCG64(seed))
    radii = np.exp(sigma * rng.standard_normal(bubbles))
    box = spacing * bubbles ** (1.0 / 3.0)
    centres = _place_centres(radii, box, gap, rng)
    mesh = cluster(level, radii, centres)
    mesh.meta.update({"seed": seed, "level": level, "box": box, "sigma": sigma, "gap": gap})
    phi = cluster_potential(mesh, phi_lmax, phi_scale, rng, radius_scaled=phi_radius_scaled)
    return mesh, phi


def workload_uneven_clusters(n_clusters: int = 64, seed: int = 5, max_bubbles: int = 200,
                             levels=(2, 3, 4)) -> list[tuple[Mesh, np.ndarray]]:
    """Independent clusters of uneven size: bubble count uniform in 1..max_bubbles, each
    bubble's icosphere level drawn uniformly from `levels`."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(n_clusters):
        nb = int(rng.integers(1, max_bubbles + 1))
        radii = np.exp(0.3 * rng.standard_normal(nb))
        box = max(4.0 * nb ** (1.0 / 3.0), 4.0 * radii.max())
        centres = _place_centres(radii, box, 0.5, rng)
        lev = rng.choice(np.asarray(levels), size=nb)
        mesh = cluster(lev, radii, centres)
        phi = cluster_potential(mesh, 6, 0.01, rng, radius_scaled=True)
        out.append((mesh, phi))
    return out


def concat_meshes(meshes, phis=None):
    """Concatenate independent meshes (e.g. separate clusters) into one Mesh; returns
    (mesh, phi or None, bubble_off) where cluster c owns bubbles bubble_off[c]..bubble_off[c+1]-1."""
    xs, ts, voff, toff, boff, cen, rad = [], [], [0], [0], [0], [], []
    for m in meshes:
        ts.append(m.tri + voff[-1])
        xs.append(m.xyz)
        for b in range(m.m):
            voff.append(voff[-1] + int(m.vert_off[b + 1] - m.vert_off[b]))
            toff.append(toff[-1] + int(m.tri_off[b + 1] - m.tri_off[b]))
        boff.append(boff[-1] + m.m)
        cen.append(m.centres)
        rad.append(m.radii)
    mesh = Mesh(xyz=np.ascontiguousarray(np.concatenate(xs)), tri=np.ascontiguousarray(np.concatenate(ts), np.int32),
                vert_off=np.asarray(voff, np.int64), tri_off=np.asarray(toff, np.int64),
                centres=np.concatenate(cen), radii=np.concatenate(rad), meta={"kind": "clusters", "clusters": len(meshes)})
    phi = None if phis is None else np.ascontiguousarray(np.concatenate(phis))
    return mesh, phi, np.asarray(boff, np.int64)

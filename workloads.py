"""Seeded synthetic meshes and vectors for the EFIE impedance-matrix fill.

This module only generates inputs: vertex coordinates (float64, units of the
free-space wavelength lambda = 1), triangle vertex indices (int32, counter-
clockwise seen from outside for closed surfaces) and seeded complex vectors.
It holds none of the fill's arithmetic, so both the CUDA library and the CPU
oracle can be fed from it.

The paper measures on a PEC sphere of radius 0.5 lambda (Section IV.B) and an
IC inductor whose geometry is not published (Section IV.B, last paragraph);
the shapes below stand in for those workloads at the sizes listed in
``CONFIGS``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TWO_PI = 2.0 * math.pi


# ----------------------------------------------------------------------------
# basic shapes
# ----------------------------------------------------------------------------
def plate(side: float = 0.5, n: int = 10, z: float = 0.0):
    """Square plate [0, side]^2 at height z, n x n squares, each split along
    the same diagonal (lower-left to upper-right) into two triangles."""
    xs = np.linspace(0.0, side, n + 1)
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    xyz = np.stack([X.ravel(), Y.ravel(), np.full(X.size, z)], axis=1)
    tris = []
    for j in range(n):
        for i in range(n):
            v00 = j * (n + 1) + i
            v10 = v00 + 1
            v01 = v00 + (n + 1)
            v11 = v01 + 1
            tris.append((v00, v10, v11))
            tris.append((v00, v11, v01))
    return xyz.astype(np.float64), np.asarray(tris, dtype=np.int32)


def _subdivide(xyz, tris, levels, radius):
    """Midpoint subdivision, projecting new vertices onto the sphere."""
    xyz = [tuple(v) for v in xyz]
    for _ in range(levels):
        cache = {}
        out = []

        def mid(a, b):
            key = (a, b) if a < b else (b, a)
            if key in cache:
                return cache[key]
            p = np.add(xyz[a], xyz[b]) * 0.5
            p = p / np.linalg.norm(p) * radius
            xyz.append(tuple(p))
            cache[key] = len(xyz) - 1
            return cache[key]

        for a, b, c in tris:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            out += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        tris = out
    return np.asarray(xyz, dtype=np.float64), np.asarray(tris, dtype=np.int32)


def icosphere(levels: int, radius: float = 1.0):
    """Icosahedron refined ``levels`` times: 20 * 4**levels triangles."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
                  (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
                  (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)], dtype=np.float64)
    v = v / np.linalg.norm(v, axis=1, keepdims=True) * radius
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
         (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
         (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
         (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    return _subdivide(v, f, levels, radius)


def octasphere(levels: int, radius: float = 1.0):
    """Octahedron refined ``levels`` times: 8 * 4**levels triangles."""
    v = np.array([(1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)],
                 dtype=np.float64) * radius
    f = [(0, 2, 4), (2, 1, 4), (1, 3, 4), (3, 0, 4),
         (2, 0, 5), (1, 2, 5), (3, 1, 5), (0, 3, 5)]
    return _subdivide(v, f, levels, radius)


def mean_edge_length(xyz, tris):
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]])
    return float(np.linalg.norm(xyz[e[:, 0]] - xyz[e[:, 1]], axis=1).mean())


def jitter(xyz, tris, frac: float, seed: int):
    """Add U[-frac*l, frac*l] to every coordinate, l = mean edge length."""
    rng = np.random.default_rng(seed)
    l = mean_edge_length(xyz, tris)
    return xyz + rng.uniform(-frac * l, frac * l, size=xyz.shape)


def uv_ellipsoid(a: float, b: float, c: float, n_theta_rings: int, n_phi: int,
                 rng: np.random.Generator, perturb: float = 0.05):
    """Closed UV ellipsoid with pole fans: 2 * n_phi * (n_theta_rings) triangles
    where n_theta_rings = (number of latitude rings + 1). The radius is scaled
    by 1 + perturb * xi(theta, phi), xi a seeded sum of 3 low-order sines
    (|xi| <= 1)."""
    terms = [(int(rng.integers(1, 4)), int(rng.integers(1, 4)), float(rng.uniform(0, TWO_PI)))
             for _ in range(3)]

    def xi(th, ph):
        return sum(math.sin(p * th + q * ph + s) for p, q, s in terms) / 3.0

    nt = n_theta_rings
    verts = [(0.0, 0.0, c * (1 + perturb * xi(0.0, 0.0)))]
    for i in range(1, nt):
        th = math.pi * i / nt
        for j in range(n_phi):
            ph = TWO_PI * j / n_phi
            s = 1 + perturb * xi(th, ph)
            verts.append((a * s * math.sin(th) * math.cos(ph),
                          b * s * math.sin(th) * math.sin(ph),
                          c * s * math.cos(th)))
    verts.append((0.0, 0.0, -c * (1 + perturb * xi(math.pi, 0.0))))
    south = len(verts) - 1

    def ring(i, j):
        return 1 + (i - 1) * n_phi + (j % n_phi)

    tris = []
    for j in range(n_phi):
        tris.append((0, ring(1, j), ring(1, j + 1)))
    for i in range(1, nt - 1):
        for j in range(n_phi):
            a0, a1 = ring(i, j), ring(i, j + 1)
            b0, b1 = ring(i + 1, j), ring(i + 1, j + 1)
            tris.append((a0, b0, b1))
            tris.append((a0, b1, a1))
    for j in range(n_phi):
        tris.append((south, ring(nt - 1, j + 1), ring(nt - 1, j)))
    return np.asarray(verts, dtype=np.float64), np.asarray(tris, dtype=np.int32)


def cube(side: float = 3.0, n: int = 64):
    """Closed cube [-side/2, side/2]^3 with n x n squares per face (welded
    edge vertices), each square split into two triangles, outward normals."""
    h = side / 2.0
    index = {}
    verts = []

    def vid(p):
        key = tuple(int(round((x + h) / side * n)) for x in p)
        if key not in index:
            index[key] = len(verts)
            verts.append(tuple(-h + k * side / n for k in key))
        return index[key]

    tris = []
    # each face: origin, u axis, v axis with u x v = outward normal
    faces = [((h, -h, -h), (0, 1, 0), (0, 0, 1)), ((-h, -h, -h), (0, 0, 1), (0, 1, 0)),
             ((-h, h, -h), (0, 0, 1), (1, 0, 0)), ((-h, -h, -h), (1, 0, 0), (0, 0, 1)),
             ((-h, -h, h), (1, 0, 0), (0, 1, 0)), ((-h, -h, -h), (0, 1, 0), (1, 0, 0))]
    d = side / n
    for o, u, v in faces:
        o, u, v = np.array(o), np.array(u), np.array(v)
        for j in range(n):
            for i in range(n):
                p00 = vid(o + u * i * d + v * j * d)
                p10 = vid(o + u * (i + 1) * d + v * j * d)
                p01 = vid(o + u * i * d + v * (j + 1) * d)
                p11 = vid(o + u * (i + 1) * d + v * (j + 1) * d)
                tris.append((p00, p10, p11))
                tris.append((p00, p11, p01))
    return np.asarray(verts, dtype=np.float64), np.asarray(tris, dtype=np.int32)


def complex_gaussian(n: int, seed: int):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(n) + 1j * rng.standard_normal(n)) / math.sqrt(2.0)


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    xyz: np.ndarray
    tri: np.ndarray
    k: float
    rule: int
    near_dist: float = 0.0        # 0: vertex-sharing pairs only
    precision: str = "fp32"
    extra: dict = field(default_factory=dict)


def plate_280():
    """PEC plate 0.5 x 0.5 lambda, 10 x 10 squares -> 200 triangles, 280 RWG."""
    xyz, tri = plate(0.5, 10)
    return Workload("plate_0.5lambda_200tri_280rwg_3pt_fp64", xyz, tri, TWO_PI, 3,
                    precision="fp64")


def sphere_7680():
    """PEC sphere r = 1 lambda, icosphere level 4 (5120 triangles, 7680 RWG),
    vertices jittered by U[+-2%] of the mean edge length, 7-point rule."""
    xyz, tri = icosphere(4, 1.0)
    xyz = jitter(xyz, tri, 0.02, 20190114)
    return Workload("sphere_r1lambda_5120tri_7680rwg_7pt_fp32", xyz, tri, TWO_PI, 7, extra={"sphere_radius": 1.0})


def sphere_3072():
    """PEC sphere r = 1 lambda, octasphere level 4 (2048 triangles, 3072 RWG),
    jittered as above, 6-point rule (adjoint workload)."""
    xyz, tri = octasphere(4, 1.0)
    xyz = jitter(xyz, tri, 0.02, 20190115)
    return Workload("sphere_r1lambda_2048tri_3072rwg_6pt_adjoint", xyz, tri, TWO_PI, 6,
                    extra={"sphere_radius": 1.0})


def cube_73728(n: int = 64):
    """PEC cube of side 3 lambda, n x n squares per face (n = 64: 49152
    triangles, 73728 RWG), 4-point rule, near pairs: centroid < 0.2 lambda."""
    xyz, tri = cube(3.0, n)
    return Workload(f"cube_3lambda_{12 * n * n}tri_{18 * n * n}rwg_4pt_fp32", xyz, tri,
                    TWO_PI, 4, near_dist=0.2)


def ellipsoid_batch(count: int = 64, first_seed: int = 1000):
    """Perturbed ellipsoids, semi-axes U[0.5, 2] lambda, target triangle
    count U[500, 4000], own k ~ U[pi, 4 pi] each, 6-point rule."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(first_seed + i)
        a, b, c = rng.uniform(0.5, 2.0, size=3)
        target = rng.uniform(500, 4000)
        k = float(rng.uniform(math.pi, 4 * math.pi))
        rings = max(2, int(round(math.sqrt(target / 4.0))) + 1)
        nphi = max(3, int(round(target / (2 * (rings - 1)))))
        xyz, tri = uv_ellipsoid(a, b, c, rings, nphi, rng)
        out.append(Workload(f"ellipsoid_{i}_{len(tri)}tri", xyz, tri, k, 6))
    return out

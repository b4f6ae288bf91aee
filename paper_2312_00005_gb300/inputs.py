"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds only input generation: surface meshes (node coordinates and
counter-clockwise triangles), field points, sources, admittances and random
vectors.  It contains none of the method's arithmetic (no normals, areas,
kernels or quadrature), so the CUDA path and the oracle can both be fed from
it without sharing any of the method.

Workloads follow the shapes the paper benchmarks (Sec. 5.1: icosahedron-based
sphere meshes; Sec. 5.2: a head-like closed surface; Sec. 5.3: a closed duct
for the interior problem) with the sizes of the configurations this library
is measured on.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "icosahedron", "icosphere", "geodesic_sphere", "bumpy_ellipsoid", "duct", "fibonacci_sphere",
    "random_complex", "workload",
]


def icosahedron():
    """Unit icosahedron: 12 vertices, 20 counter-clockwise (outward) faces."""
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([
        [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
        [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
        [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1],
    ], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
    ], dtype=np.int32)
    return v, f


def _orient_outward(nodes, tris):
    """Flip faces whose winding points toward the origin (star-shaped surfaces)."""
    a, b, c = nodes[tris[:, 0]], nodes[tris[:, 1]], nodes[tris[:, 2]]
    s = np.einsum("ij,ij->i", np.cross(b - a, c - a), a + b + c)
    bad = s < 0
    tris = tris.copy()
    tris[bad] = tris[bad][:, [0, 2, 1]]
    return tris


def icosphere(level: int, radius: float = 1.0):
    """Icosahedron split `level` times into 4 (edge midpoints), projected onto
    the sphere: N = 20 * 4**level triangles (the paper's icosahedron meshes,
    Sec. 5.1).  Returns (nodes float64 [Nv,3], tris int32 [N,3])."""
    v, f = icosahedron()
    verts = [tuple(x) for x in v]
    nodes = list(v)
    for _ in range(level):
        cache = {}

        def mid(i, j):
            key = (min(i, j), max(i, j))
            if key not in cache:
                m = 0.5 * (nodes[i] + nodes[j])
                m = m / np.linalg.norm(m)
                cache[key] = len(nodes)
                nodes.append(m)
            return cache[key]

        nf = []
        for (a, b, c) in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca)]
        f = np.array(nf, dtype=np.int32)
    del verts
    nodes = np.array(nodes, dtype=np.float64) * radius
    return nodes, _orient_outward(nodes, np.ascontiguousarray(f, dtype=np.int32))


def geodesic_sphere(nu: int):
    """Class-I geodesic sphere of frequency nu: each icosahedron face cut into
    nu*nu triangles, vertices projected on the unit sphere (N = 20 nu^2)."""
    v, f = icosahedron()
    index = {}
    nodes = []

    def vid(p):
        q = p / np.linalg.norm(p)
        key = tuple(np.round(q * 1e9).astype(np.int64))
        if key not in index:
            index[key] = len(nodes)
            nodes.append(q)
        return index[key]

    tris = []
    for (a, b, c) in f:
        A, B, C = v[a], v[b], v[c]
        grid = {}
        for i in range(nu + 1):
            for j in range(nu + 1 - i):
                p = A + (B - A) * (i / nu) + (C - A) * (j / nu)
                grid[(i, j)] = vid(p)
        for i in range(nu):
            for j in range(nu - i):
                tris.append((grid[(i, j)], grid[(i + 1, j)], grid[(i, j + 1)]))
                if i + j < nu - 1:
                    tris.append((grid[(i + 1, j)], grid[(i + 1, j + 1)], grid[(i, j + 1)]))
    nodes = np.array(nodes, dtype=np.float64)
    tris = np.array(tris, dtype=np.int32)
    return nodes, _orient_outward(nodes, tris)


def bumpy_ellipsoid(nu: int, axes=(0.09, 0.075, 0.11), n_bumps: int = 24, seed: int = 2312,
                    amp=(0.002, 0.006), sigma=(0.15, 0.35)):
    """Head-like closed surface: geodesic sphere of frequency nu mapped onto an
    ellipsoid with the given semi-axes, plus seeded smooth Gaussian radial bumps
    (amplitude and angular width drawn uniformly from the given ranges)."""
    u, tris = geodesic_sphere(nu)
    nodes = _head_map(u, axes, n_bumps, seed, amp, sigma)
    return nodes, _orient_outward(nodes, tris)


def _head_map(u, axes=(0.09, 0.075, 0.11), n_bumps=24, seed=2312, amp=(0.002, 0.006), sigma=(0.15, 0.35)):
    """The head-like surface as a map of unit vectors u [M, 3]: ellipsoid
    point plus the seeded radial bumps."""
    rng = np.random.default_rng(seed)
    cen = rng.normal(size=(n_bumps, 3))
    cen /= np.linalg.norm(cen, axis=1, keepdims=True)
    a = rng.uniform(amp[0], amp[1], n_bumps)
    s = rng.uniform(sigma[0], sigma[1], n_bumps)
    e = u * np.asarray(axes, dtype=np.float64)[None, :]
    ang = np.arccos(np.clip(u @ cen.T, -1.0, 1.0))
    disp = (a[None, :] * np.exp(-0.5 * (ang / s[None, :]) ** 2)).sum(axis=1)
    return e + disp[:, None] * u


def head_point_source(offset: float = 0.001):
    """Position of the batched-frequency workload's point source: offset
    metres outside the head-like surface at the image of +y (its +y
    extremum), along +y."""
    y = _head_map(np.array([[0.0, 1.0, 0.0]]))[0]
    return y + np.array([0.0, offset, 0.0])


def head_bands(n_freq: int = 64, f_lo: float = 200.0, f_hi: float = 16000.0, c: float = 343.0,
               per_wavelength: float = 10.7, h_max: float = 0.011, step: float = 1.15):
    """The batched-frequency workload on the head-like surface: n_freq
    frequencies f_i = f_lo (f_hi / f_lo)^(i / (n_freq - 1)), each wanting a
    mean element edge h_i = min(lambda_i / per_wavelength, h_max).  The mean
    edge of bumpy_ellipsoid(nu) is kappa / nu (kappa measured on nu = 10);
    each frequency takes the smallest nu of the ladder ceil(nu_0 step^j)
    with kappa / nu <= h_i, so frequencies share meshes in bands of uneven
    N = 20 nu^2.  Returns [(nu, [freqs])] in increasing frequency."""
    nodes, tris = bumpy_ellipsoid(10)
    e = np.concatenate([np.linalg.norm(nodes[tris[:, a]] - nodes[tris[:, b]], axis=1)
                        for a, b in ((0, 1), (1, 2), (2, 0))])
    kappa = float(e.mean()) * 10
    freqs = f_lo * (f_hi / f_lo) ** (np.arange(n_freq) / (n_freq - 1))
    need = np.ceil(kappa / np.minimum(c / freqs / per_wavelength, h_max)).astype(int)
    ladder = [int(need.min())]
    while ladder[-1] < need.max():
        ladder.append(max(ladder[-1] + 1, int(np.ceil(ladder[0] * step ** len(ladder)))))
    bands = []
    for f, nd in zip(freqs, need):
        nu = next(v for v in ladder if v >= nd)
        if bands and bands[-1][0] == nu:
            bands[-1][1].append(float(f))
        else:
            bands.append((nu, [float(f)]))
    return bands


def duct(length: float = 3.4, width: float = 0.2, h: float = 0.05):
    """Closed duct [0, length] x [-width/2, width/2]^2 (the paper's duct
    benchmark, Sec. 5.3): every face cut into squares of edge about h, each
    square into two triangles, wound so that (b - a) x (c - a) points out of
    the enclosed volume.  Returns (nodes float64 [Nv,3], tris int32 [N,3])."""
    nx = max(1, int(round(length / h)))
    ny = max(1, int(round(width / h)))
    xs = np.linspace(0.0, length, nx + 1)
    ys = np.linspace(-width / 2, width / 2, ny + 1)
    centre = np.array([length / 2, 0.0, 0.0])
    nodes, tris = [], []

    def face(us, vs, point):
        base = len(nodes)
        for u in us:
            for v in vs:
                nodes.append(point(u, v))
        m = len(vs)
        for a in range(len(us) - 1):
            for b in range(m - 1):
                i00, i01 = base + a * m + b, base + a * m + b + 1
                i10, i11 = base + (a + 1) * m + b, base + (a + 1) * m + b + 1
                tris.append([i00, i10, i11])
                tris.append([i00, i11, i01])

    face(ys, ys, lambda u, v: (0.0, u, v))
    face(ys, ys, lambda u, v: (length, u, v))
    face(xs, ys, lambda u, v: (u, -width / 2, v))
    face(xs, ys, lambda u, v: (u, width / 2, v))
    face(xs, ys, lambda u, v: (u, v, -width / 2))
    face(xs, ys, lambda u, v: (u, v, width / 2))
    nodes = np.array(nodes, dtype=np.float64)
    tris = np.array(tris, dtype=np.int32)
    a, b, c = nodes[tris[:, 0]], nodes[tris[:, 1]], nodes[tris[:, 2]]
    out = np.einsum("ij,ij->i", np.cross(b - a, c - a), (a + b + c) / 3.0 - centre) < 0
    tris[out] = tris[out][:, [0, 2, 1]]
    return nodes, tris


def fibonacci_sphere(m: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """m points spread on a sphere by the Fibonacci lattice."""
    i = np.arange(m, dtype=np.float64) + 0.5
    z = 1.0 - 2.0 * i / m
    phi = math.pi * (3.0 - 5.0 ** 0.5) * i
    r = np.sqrt(1.0 - z * z)
    p = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1) * radius
    return p + np.asarray(center, dtype=np.float64)[None, :]


def random_complex(n: int, seed: int, shape=None):
    """Seeded complex128 vector (standard normal real and imaginary parts)."""
    rng = np.random.default_rng(seed)
    shp = (n,) if shape is None else shape
    return rng.normal(size=shp) + 1j * rng.normal(size=shp)


def tetrahedral_directions():
    """The four unit directions (+-1, +-1, +-1) / sqrt(3) with an even number
    of minus signs (the vertices of a regular tetrahedron)."""
    d = np.array([[1.0, 1.0, 1.0], [1.0, -1.0, -1.0], [-1.0, 1.0, -1.0], [-1.0, -1.0, 1.0]])
    return d / np.sqrt(3.0)


def workload(name: str):
    """The synthetic workloads the library is checked and measured on.

    sphere1280_1k  : sound-hard sphere r = 0.1 m, icosphere of 1280 triangles,
                     plane wave along +z at 1 kHz (small oracle case).
    sphere5120_2k  : the same sphere as an icosphere of 5120 triangles at 2 kHz.
    sphere20480_4k : the same sphere as an icosphere of 20480 triangles, plane
                     wave along +z at 4 kHz, 100 field points on a 1 m sphere.
    bumpy158k_20k  : the head-like bumpy ellipsoid (bumpy_ellipsoid) at
                     geodesic frequency 89 (158420 triangles, mean edge 1.3 mm,
                     about a thirteenth of the wavelength) at 20 kHz, four
                     plane waves along the tetrahedral directions (one
                     right-hand side each).
    """
    if name == "sphere1280_1k":
        nodes, tris = icosphere(3, 0.1)
        freq = 1000.0
    elif name == "sphere5120_2k":
        nodes, tris = icosphere(4, 0.1)
        freq = 2000.0
    elif name == "sphere20480_4k":
        nodes, tris = icosphere(5, 0.1)
        freq = 4000.0
    elif name == "bumpy158k_20k":
        nodes, tris = bumpy_ellipsoid(89)
        freq = 20000.0
    else:
        raise KeyError(name)
    out = {
        "name": name, "nodes": nodes, "tris": tris, "freq": freq, "c": 343.0, "rho": 1.21,
        "plane_dir": (0.0, 0.0, 1.0), "amp": 1.0 + 0.0j,
        "field_points": fibonacci_sphere(100, 1.0),
    }
    if name == "bumpy158k_20k":
        out["plane_dirs"] = tetrahedral_directions()
    return out

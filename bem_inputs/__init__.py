"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module only builds inputs: surface grids (icospheres, rotated and jittered
copies, ellipsoids), incident-wave directions and request streams.  It holds none
of the boundary element arithmetic.  Grids stand in for the Gmsh meshes of the
paper (unit cube, screen and foam of Sec. 5), which are not available; the
workloads are the sphere and ellipsoid cases of the transmission benchmark.

Conventions
-----------
* vertices: float64 array [N, 3]; triangles: int32 array [T, 3], counter-clockwise
  seen from outside, so that (b - a) x (c - a) points outward (Sec. 2: the normal is
  always the outward one).
* every random draw takes an explicit integer seed (numpy PCG64).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "icosphere",
    "haar_rotation",
    "rotate_and_jitter",
    "ellipsoid",
    "transmission_pair",
    "plane_wave_directions",
    "unit_square_grid",
    "perturb_square_grid",
    "cube_grid",
    "screen_grid",
    "disk_grid",
    "serving_requests",
]


def _icosahedron():
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array(
        [
            [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
            [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
            [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1],
        ],
        dtype=np.float64,
    )
    f = np.array(
        [
            [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
            [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
            [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
            [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1],
        ],
        dtype=np.int64,
    )
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v, f


def _orient_outward(v, f):
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    nrm = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", nrm, (a + b + c) / 3.0) < 0
    f = f.copy()
    f[flip, 1], f[flip, 2] = f[flip, 2].copy(), f[flip, 1].copy()
    return f


def icosphere(level: int):
    """Unit icosphere by `level` midpoint 4-splits of the icosahedron.

    Returns (vertices f64[N,3], triangles i32[T,3]) with N = 10*4**level + 2 and
    T = 20*4**level; triangles are oriented outward.
    """
    if level < 0:
        raise ValueError("level must be >= 0")
    v, f = _icosahedron()
    verts = [tuple(x) for x in v]
    vlist = list(v)
    for _ in range(level):
        cache = {}
        nf = []

        def mid(i, j):
            key = (i, j) if i < j else (j, i)
            if key in cache:
                return cache[key]
            m = (vlist[i] + vlist[j]) * 0.5
            m = m / np.linalg.norm(m)
            vlist.append(m)
            cache[key] = len(vlist) - 1
            return cache[key]

        for a, b, c in f:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [[a, ab, ca], [b, bc, ab], [c, ca, bc], [ab, bc, ca]]
        f = np.array(nf, dtype=np.int64)
    del verts
    v = np.array(vlist, dtype=np.float64)
    f = _orient_outward(v, f)
    return v, f.astype(np.int32)


def haar_rotation(seed: int):
    """Rotation matrix drawn from the Haar measure on SO(3) (unit quaternion of
    four i.i.d. standard normals)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array(
        [
            [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
            [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
            [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
        ]
    )


def mean_edge_length(v, f):
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
    e = np.unique(np.sort(e, axis=1), axis=0)
    return float(np.mean(np.linalg.norm(v[e[:, 0]] - v[e[:, 1]], axis=1)))


def rotate_and_jitter(v, f, seed: int, jitter: float = 0.01):
    """Nonconforming copy of a unit-sphere grid.

    1. rotate by a Haar-random rotation (seed);
    2. move every vertex by jitter * (mean edge length) along a uniformly random
       tangent direction (seed + 1000003);
    3. project back onto the unit sphere.
    """
    R = haar_rotation(seed)
    w = v @ R.T
    h = mean_edge_length(w, f)
    rng = np.random.Generator(np.random.PCG64(seed + 1000003))
    d = rng.standard_normal(w.shape)
    d -= np.einsum("ij,ij->i", d, w)[:, None] * w
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    w = w + jitter * h * d
    w /= np.linalg.norm(w, axis=1, keepdims=True)
    return w


def ellipsoid(v, axes):
    """Scale unit-sphere vertices by diag(a, b, c); orientation is preserved."""
    return v * np.asarray(axes, dtype=np.float64)[None, :]


def transmission_pair(level_ext: int, level_int: int, seed: int, axes=None, jitter: float = 0.01):
    """Exterior grid = plain icosphere; interior grid = icosphere rotated and
    jittered (nonconforming).  Both are scaled onto the ellipsoid `axes` last.

    Returns (v_ext, t_ext, v_int, t_int)."""
    ve, te = icosphere(level_ext)
    vi, ti = icosphere(level_int)
    vi = rotate_and_jitter(vi, ti, seed, jitter)
    if axes is not None:
        ve = ellipsoid(ve, axes)
        vi = ellipsoid(vi, axes)
    return ve, te, vi, ti


def plane_wave_directions(n: int, seed: int):
    """n unit vectors uniform on S^2 (normalised standard normal draws)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    d = rng.standard_normal((n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def unit_square_grid(n: int):
    """Structured triangulation of [0,1]^2 (z = 0) with (n+1)^2 nodes, normal +z."""
    x = np.linspace(0.0, 1.0, n + 1)
    X, Y = np.meshgrid(x, x, indexing="ij")
    v = np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)
    idx = lambda i, j: i * (n + 1) + j
    tri = []
    for i in range(n):
        for j in range(n):
            a, b, c, d = idx(i, j), idx(i + 1, j), idx(i + 1, j + 1), idx(i, j + 1)
            if (i + j) % 2 == 0:
                tri += [[a, b, c], [a, c, d]]
            else:
                tri += [[a, b, d], [b, c, d]]
    return v, np.array(tri, dtype=np.int32)


def cube_grid(n: int, jitter: float = 0.0, seed: int = 0):
    """Surface of the unit cube [0,1]^3 (the geometry of the accuracy and efficiency
    benchmarks of Sec. 5.3-5.5) with each face a structured n x n grid of squares cut
    into two triangles (diagonals alternating), faces sharing their edge nodes, so the
    surface grid is conforming with 6 n^2 + 2 nodes.  jitter > 0 moves the nodes
    inside each face (not those on cube edges) by a seeded uniform offset of at most
    jitter * (1/n) along each in-face axis, so two grids of one size still differ.
    Triangles are counter-clockwise seen from outside."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h = 1.0 / n
    index = {}
    verts = []

    def node(p):
        key = tuple(int(c) for c in p)
        if key not in index:
            index[key] = len(verts)
            verts.append(key)
        return index[key]

    tris = []
    for axis in range(3):
        u, w = [a for a in range(3) if a != axis]
        for side in (0, n):
            ids = np.empty((n + 1, n + 1), dtype=np.int64)
            for i in range(n + 1):
                for j in range(n + 1):
                    p = [0, 0, 0]
                    p[axis], p[u], p[w] = side, i, j
                    ids[i, j] = node(p)
            for i in range(n):
                for j in range(n):
                    a, b, c, d = ids[i, j], ids[i + 1, j], ids[i + 1, j + 1], ids[i, j + 1]
                    if (i + j) % 2 == 0:
                        tris += [[a, b, c], [a, c, d]]
                    else:
                        tris += [[a, b, d], [b, c, d]]
    lat = np.array(verts, dtype=np.float64)
    v = lat * h
    if jitter > 0.0:
        on_edge = ((lat == 0) | (lat == n)).sum(axis=1) >= 2
        off = rng.uniform(-jitter * h, jitter * h, size=v.shape)
        face_axis = np.argmax((lat == 0) | (lat == n), axis=1)
        off[np.arange(len(v)), face_axis] = 0.0
        off[on_edge] = 0.0
        v = v + off
    f = np.array(tris, dtype=np.int64)
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    nrm = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", nrm, (a + b + c) / 3.0 - 0.5) < 0
    f[flip, 1], f[flip, 2] = f[flip, 2].copy(), f[flip, 1].copy()
    return v, f.astype(np.int32)


# Corners of the rectangular screen of the operator-preconditioning benchmark (Sec. 5.7):
# edge lengths about 2.06 (first direction) and 2.
SCREEN_CORNERS = ((-0.25, -1.0, -1.0), (0.25, 1.0, -1.0), (0.25, 1.0, 1.0), (-0.25, -1.0, 1.0))


def screen_grid(nu: int, nv: int, jitter: float = 0.0, seed: int = 0):
    """Open rectangular screen with corners SCREEN_CORNERS (c0, c1, c2, c3), a structured
    nu x nv grid of cells along c1 - c0 and c3 - c0 cut into two triangles each
    (diagonals alternating), (nu + 1)(nv + 1) nodes.  jitter > 0 moves the nodes that are
    not on the boundary by a seeded uniform in-plane offset of at most jitter cell widths
    along each direction.  Every triangle is oriented like (c1 - c0) x (c3 - c0)."""
    c0, c1, _, c3 = (np.asarray(c, dtype=np.float64) for c in SCREEN_CORNERS)
    eu, ev = c1 - c0, c3 - c0
    s = np.linspace(0.0, 1.0, nu + 1)
    t = np.linspace(0.0, 1.0, nv + 1)
    S, T = np.meshgrid(s, t, indexing="ij")
    S, T = S.ravel().copy(), T.ravel().copy()
    if jitter > 0.0:
        rng = np.random.Generator(np.random.PCG64(seed))
        inner = (S > 0) & (S < 1) & (T > 0) & (T < 1)
        S[inner] += rng.uniform(-jitter / nu, jitter / nu, inner.sum())
        T[inner] += rng.uniform(-jitter / nv, jitter / nv, inner.sum())
    v = c0[None, :] + S[:, None] * eu[None, :] + T[:, None] * ev[None, :]
    idx = lambda i, j: i * (nv + 1) + j
    tri = []
    for i in range(nu):
        for j in range(nv):
            a, b, c, d = idx(i, j), idx(i + 1, j), idx(i + 1, j + 1), idx(i, j + 1)
            if (i + j) % 2 == 0:
                tri += [[a, b, c], [a, c, d]]
            else:
                tri += [[a, b, d], [b, c, d]]
    return v, np.array(tri, dtype=np.int32)


def disk_grid(n: int):
    """The unit disk in the plane z = 0 as a ring grid: the centre and n rings of radius
    k/n with 6k nodes each (1 + 3n(n + 1) nodes, 6n^2 triangles), neighbouring rings
    joined in order of angle; every triangle is counter-clockwise seen from +z."""
    pts = [(0.0, 0.0)]
    rings = [[0]]
    for k in range(1, n + 1):
        m = 6 * k
        ids = []
        for q in range(m):
            th = 2.0 * np.pi * q / m
            ids.append(len(pts))
            pts.append((k / n * np.cos(th), k / n * np.sin(th)))
        rings.append(ids)
    tri = [(0, rings[1][q], rings[1][(q + 1) % 6]) for q in range(6)]
    for k in range(2, n + 1):
        inner, outer = rings[k - 1], rings[k]
        mi, mo = len(inner), len(outer)
        i = j = 0
        while i < mi or j < mo:
            if j < mo and (i >= mi or (j + 1) * mi <= (i + 1) * mo):
                tri.append((inner[i % mi], outer[j % mo], outer[(j + 1) % mo]))
                j += 1
            else:
                tri.append((inner[i % mi], outer[j % mo], inner[(i + 1) % mi]))
                i += 1
    v = np.array([(x, y, 0.0) for x, y in pts])
    t = np.array(tri, dtype=np.int64)
    a, b, c = v[t[:, 0]], v[t[:, 1]], v[t[:, 2]]
    flip = np.cross(b - a, c - a)[:, 2] < 0
    t[flip, 1], t[flip, 2] = t[flip, 2].copy(), t[flip, 1].copy()
    return v, t.astype(np.int32)


def perturb_square_grid(v, sigma: float, seed: int):
    """Gaussian node perturbation of a unit-square grid with N(0, sigma): interior
    nodes move in both directions, boundary nodes only along the boundary, corners
    not at all (the perturbation experiment of Sec. 5.2).  Perturbations are
    clipped so that no node leaves the square or passes a neighbour."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = v.copy()
    d = rng.standard_normal((len(v), 2)) * sigma
    eps = 1e-12
    on_x = (np.abs(v[:, 0]) < eps) | (np.abs(v[:, 0] - 1) < eps)
    on_y = (np.abs(v[:, 1]) < eps) | (np.abs(v[:, 1] - 1) < eps)
    d[on_x, 0] = 0.0
    d[on_y, 1] = 0.0
    w[:, :2] += d
    w[:, :2] = np.clip(w[:, :2], 0.0, 1.0)
    return w


def serving_requests(n: int, seed: int, rate: float):
    """Poisson-arrival stream of transmission requests (the serving workload):
    ellipsoid semi-axes ~ U[0.5,1.5]^3, independent ext/int icosphere levels in
    {2,3,4}, k_ext ~ U[1,8], k_int/k_ext ~ U[1.2,2], rho_int/rho_ext log-uniform on
    [0.1,10], 1-16 plane waves.  `rate` is arrivals per second.  Arrival gaps and
    request parameters come from two generators drawn in request order, so the
    first n requests of a longer stream are the same requests."""
    rng_t = np.random.Generator(np.random.PCG64([seed, 0]))
    rng = np.random.Generator(np.random.PCG64([seed, 1]))
    t = np.cumsum(rng_t.exponential(1.0 / rate, size=n))
    reqs = []
    for i in range(n):
        axes = rng.uniform(0.5, 1.5, size=3)
        le, li = int(rng.integers(2, 5)), int(rng.integers(2, 5))
        k_ext = float(rng.uniform(1.0, 8.0))
        k_int = k_ext * float(rng.uniform(1.2, 2.0))
        rho = float(np.exp(rng.uniform(np.log(0.1), np.log(10.0))))
        nrhs = int(rng.integers(1, 17))
        dirs = rng.standard_normal((nrhs, 3))
        dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        reqs.append(
            dict(arrival=float(t[i]), axes=axes, level_ext=le, level_int=li, k_ext=k_ext,
                 k_int=k_int, rho_ratio=rho, dirs=dirs, seed=int(seed * 100003 + i))
        )
    return reqs

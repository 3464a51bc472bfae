"""Seeded synthetic inputs: surface meshes, evaluation points and field-line seeds.

This module holds no arithmetic of the boundary element method itself.  It only
builds the geometry and sample points that both the CUDA path and the CPU
oracle are fed with, so that the two can be compared on identical inputs.

Conventions (Sec. 2 of the paper, Fig. 2): every body is a closed surface made
of flat triangles; each triangle's vertices are ordered counter-clockwise when
seen from the side its normal points to, and that normal points out of the body
(into the exterior medium, the "+" side).  A thin floating sheet is a single,
possibly open surface whose normal picks its "+" side (Eq. sheets).

Region descriptors are plain dicts::

    {"kind": "conductor",  "V0": 1.0}
    {"kind": "floating",   "floating_id": 0, "eps_plus": 1.0}
    {"kind": "dielectric", "eps_plus": 1.0, "eps_minus": 4.0}
    {"kind": "sheet",      "floating_id": 1, "eps_plus": 1.0, "eps_minus": 4.0}

Floating conductors and sheets share one numbering of floating bodies.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

KIND_CODE = {"conductor": 0, "floating": 1, "dielectric": 2, "sheet": 3}
FLOATING_KINDS = ("floating", "sheet")


@dataclass
class Mesh:
    """A flat-triangle surface mesh with a region tag per triangle."""

    X: np.ndarray            # (nv, 3) float64 vertex coordinates
    tri: np.ndarray          # (np, 3) int32 vertex indices, CCW about the outward normal
    region: np.ndarray       # (np,) int32 index into ``regions``
    regions: list = field(default_factory=list)
    info: dict = field(default_factory=dict)

    @property
    def nv(self) -> int:
        return int(self.X.shape[0])

    @property
    def np_(self) -> int:
        return int(self.tri.shape[0])

    @property
    def n_floating(self) -> int:
        ids = {r["floating_id"] for r in self.regions if r["kind"] in FLOATING_KINDS}
        return len(ids)

    @property
    def n_unknowns(self) -> int:
        return self.np_ + self.n_floating


# --------------------------------------------------------------------------- helpers
def _orient_outward(X: np.ndarray, tri: np.ndarray, outward) -> np.ndarray:
    """Flip triangles whose vertex order disagrees with ``outward(centroid)``."""
    a, b, c = X[tri[:, 0]], X[tri[:, 1]], X[tri[:, 2]]
    nrm = np.cross(b - a, c - a)
    ctr = (a + b + c) / 3.0
    want = outward(ctr)
    flip = np.einsum("ij,ij->i", nrm, want) < 0
    tri = tri.copy()
    tri[flip] = tri[flip][:, [0, 2, 1]]
    return tri


def _merge(parts):
    """Concatenate (X, tri, region) parts into one mesh with shifted indices."""
    Xs, Ts, Rs, off = [], [], [], 0
    for X, tri, reg in parts:
        Xs.append(X)
        Ts.append(tri + off)
        Rs.append(np.full(len(tri), reg, dtype=np.int32))
        off += len(X)
    return np.concatenate(Xs), np.concatenate(Ts).astype(np.int32), np.concatenate(Rs)


def _icosahedron():
    """The 12 vertices and 20 faces of a regular icosahedron on the unit sphere.

    Faces are found as the triples of mutually adjacent vertices (edge length 2
    before normalisation), then oriented outward.
    """
    g = (1.0 + math.sqrt(5.0)) / 2.0
    V = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            V += [(0.0, s1, s2 * g), (s1, s2 * g, 0.0), (s2 * g, 0.0, s1)]
    V = np.array(V)
    n = len(V)
    adj = [[abs(np.linalg.norm(V[i] - V[j]) - 2.0) < 1e-9 for j in range(n)] for i in range(n)]
    F = [(i, j, k) for i in range(n) for j in range(i + 1, n) for k in range(j + 1, n)
         if adj[i][j] and adj[j][k] and adj[i][k]]
    V = V / np.linalg.norm(V, axis=1, keepdims=True)
    F = np.array(F, dtype=np.int64)
    F = _orient_outward(V, F, lambda c: c)
    return V, F


# --------------------------------------------------------------------------- bodies
def icosphere(level: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Recursively subdivided icosahedron: 20*4**level triangles on a sphere.

    Each subdivision splits a triangle into four through its edge midpoints,
    which are pushed out to the sphere.  Level 3 gives 1280 triangles and 642
    vertices.
    """
    V, F = _icosahedron()
    V = [tuple(v) for v in V]
    for _ in range(level):
        cache = {}
        newF = []

        def mid(i, j):
            key = (min(i, j), max(i, j))
            if key not in cache:
                m = (np.array(V[i]) + np.array(V[j])) / 2.0
                m = m / np.linalg.norm(m)
                V.append(tuple(m))
                cache[key] = len(V) - 1
            return cache[key]

        for a, b, c in F:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            newF += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        F = np.array(newF, dtype=np.int64)
    X = np.array(V) * radius + np.asarray(center, dtype=np.float64)
    return X, np.asarray(F, dtype=np.int32)


def geodesic_sphere(freq: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Geodesic sphere of frequency ``freq``: 20*freq**2 triangles.

    Every icosahedron face is cut into freq**2 triangles on a barycentric grid
    whose points are then projected onto the sphere.
    """
    V0, F0 = _icosahedron()
    index = {}
    V = []
    tris = []

    def vid(p):
        key = tuple(np.round(p, 10))
        if key not in index:
            index[key] = len(V)
            V.append(p / np.linalg.norm(p))
        return index[key]

    m = freq
    for a, b, c in F0:
        A, B, C = V0[a], V0[b], V0[c]
        ids = {}
        for i in range(m + 1):
            for j in range(m + 1 - i):
                k = m - i - j
                ids[(i, j)] = vid((i * A + j * B + k * C) / m)
        for i in range(m):
            for j in range(m - i):
                tris.append((ids[(i, j)], ids[(i + 1, j)], ids[(i, j + 1)]))
                if i + j < m - 1:
                    tris.append((ids[(i + 1, j)], ids[(i + 1, j + 1)], ids[(i, j + 1)]))
    X = np.array(V) * radius + np.asarray(center, dtype=np.float64)
    tri = np.array(tris, dtype=np.int64)
    c = np.asarray(center, dtype=np.float64)
    tri = _orient_outward(X, tri, lambda p: p - c)
    return X, tri.astype(np.int32)


def torus(n_u: int, n_v: int, R: float = 2.0, r: float = 0.3, z0: float = 0.0):
    """Torus with axis z: n_u cells around the axis, n_v around the tube."""
    u = 2.0 * np.pi * np.arange(n_u) / n_u
    v = 2.0 * np.pi * np.arange(n_v) / n_v
    U, Vv = np.meshgrid(u, v, indexing="ij")
    X = np.stack([(R + r * np.cos(Vv)) * np.cos(U),
                  (R + r * np.cos(Vv)) * np.sin(U),
                  r * np.sin(Vv) + z0], axis=-1).reshape(-1, 3)
    idx = lambda i, k: (i % n_u) * n_v + (k % n_v)
    tris = []
    for i in range(n_u):
        for k in range(n_v):
            p00, p10, p11, p01 = idx(i, k), idx(i + 1, k), idx(i + 1, k + 1), idx(i, k + 1)
            tris += [(p00, p10, p11), (p00, p11, p01)]
    tri = np.array(tris, dtype=np.int64)

    def outward(p):
        rho = np.hypot(p[:, 0], p[:, 1])
        core = np.stack([R * p[:, 0] / rho, R * p[:, 1] / rho, np.full(len(p), z0)], axis=-1)
        return p - core

    tri = _orient_outward(X, tri, outward)
    return X, tri.astype(np.int32)


def _ring_strip(inner, outer, ang_in, ang_out):
    """Triangulate the annulus between two closed vertex rings by a walk in angle."""
    tris = []
    ni, no = len(inner), len(outer)
    i = j = 0
    while i < ni or j < no:
        a_next_in = ang_in[i + 1] if i + 1 <= ni else np.inf
        a_next_out = ang_out[j + 1] if j + 1 <= no else np.inf
        if j < no and (i >= ni or a_next_out <= a_next_in):
            tris.append((inner[i % ni], outer[j % no], outer[(j + 1) % no]))
            j += 1
        else:
            tris.append((inner[i % ni], outer[j % no], inner[(i + 1) % ni]))
            i += 1
    return tris


def closed_cylinder(radius: float, height: float, center, K: int, n_z: int):
    """Closed cylinder (axis z): a side grid of 6K x n_z cells and two flat
    caps made of K concentric rings (ring k has 6k vertices).  The caps share
    the rim vertices with the side, so the surface is watertight."""
    cx, cy, cz = center
    n_t = 6 * K
    z = cz - height / 2.0 + height * np.arange(n_z + 1) / n_z
    th = 2.0 * np.pi * np.arange(n_t) / n_t
    X = [np.array([cx + radius * np.cos(t), cy + radius * np.sin(t), zk]) for zk in z for t in th]
    side = lambda i, k: k * n_t + (i % n_t)
    tris = []
    for k in range(n_z):
        for i in range(n_t):
            p00, p10, p11, p01 = side(i, k), side(i + 1, k), side(i + 1, k + 1), side(i, k + 1)
            tris += [(p00, p10, p11), (p00, p11, p01)]
    for cap, zc in ((0, z[0]), (n_z, z[-1])):
        centre = len(X)
        X.append(np.array([cx, cy, zc]))
        prev, prev_ang = [centre], np.array([0.0, 2.0 * np.pi])
        for k in range(1, K + 1):
            nk = 6 * k
            ang = 2.0 * np.pi * np.arange(nk) / nk
            if k == K:
                ring = [side(i, cap) for i in range(nk)]
            else:
                ring = []
                for t in ang:
                    ring.append(len(X))
                    rk = radius * k / K
                    X.append(np.array([cx + rk * np.cos(t), cy + rk * np.sin(t), zc]))
            ang_c = np.append(ang, 2.0 * np.pi)
            if k == 1:
                tris += [(centre, ring[j], ring[(j + 1) % nk]) for j in range(nk)]
            else:
                tris += _ring_strip(prev, ring, prev_ang, ang_c)
            prev, prev_ang = ring, ang_c
    X = np.array(X)
    tri = np.array(tris, dtype=np.int64)
    c = np.array(center, dtype=np.float64)

    def outward(p):
        d = p - c
        out = np.zeros_like(p)
        top = d[:, 2] > height / 2.0 - 1e-9
        bot = d[:, 2] < -height / 2.0 + 1e-9
        sid = ~(top | bot)
        out[top, 2] = 1.0
        out[bot, 2] = -1.0
        out[sid, 0], out[sid, 1] = d[sid, 0], d[sid, 1]
        return out

    tri = _orient_outward(X, tri, outward)
    return X, tri.astype(np.int32)


def open_cylinder(radius: float, z0: float, z1: float, n_t: int, n_z: int):
    """Open cylindrical sheet (axis z, no caps, z0 <= z <= z1): a grid of n_t x n_z
    cells, each split into two triangles, normals pointing away from the axis."""
    z = z0 + (z1 - z0) * np.arange(n_z + 1) / n_z
    th = 2.0 * np.pi * np.arange(n_t) / n_t
    X = np.array([[radius * np.cos(t), radius * np.sin(t), zk] for zk in z for t in th])
    side = lambda i, k: k * n_t + (i % n_t)
    tris = []
    for k in range(n_z):
        for i in range(n_t):
            p00, p10, p11, p01 = side(i, k), side(i + 1, k), side(i + 1, k + 1), side(i, k + 1)
            tris += [(p00, p10, p11), (p00, p11, p01)]
    tri = np.array(tris, dtype=np.int64)

    def outward(p):
        out = p.copy()
        out[:, 2] = 0.0
        return out

    return X, _orient_outward(X, tri, outward).astype(np.int32)


def quadratic_from_flat(X: np.ndarray, tri: np.ndarray, project=None):
    """Six-node (quadratic) triangles from a flat mesh: the corner nodes are the
    vertices X (indices 0 .. nv-1, unchanged), followed by one node per edge at the
    edge's midpoint, moved by project(points) -> points if given (e.g. onto a
    sphere).  Returns (nodes, tri6) with tri6 [N][6] = (v0, v1, v2, m01, m12, m20)."""
    tri = np.asarray(tri, dtype=np.int64)
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    key = np.sort(e, axis=1)
    uniq, inv = np.unique(key, axis=0, return_inverse=True)
    mid = 0.5 * (X[uniq[:, 0]] + X[uniq[:, 1]])
    if project is not None:
        mid = project(mid)
    n = len(tri)
    inv = inv.reshape(-1)
    m01, m12, m20 = inv[:n], inv[n:2 * n], inv[2 * n:]
    nv = len(X)
    tri6 = np.column_stack([tri, nv + m01, nv + m12, nv + m20]).astype(np.int32)
    return np.concatenate([X, mid]), tri6


def quadratic_sphere(level: int, radius: float = 1.0):
    """Icosphere of the given subdivision level as six-node triangles whose edge
    nodes lie on the sphere (piecewise quadratic parametrisation of Sec. 3).
    Returns (nodes, tri6, nv): the first nv nodes are the triangle corners."""
    X, tri = icosphere(level, radius)
    nodes, tri6 = quadratic_from_flat(
        X, tri, lambda p: radius * p / np.linalg.norm(p, axis=1, keepdims=True))
    return nodes, tri6, len(X)


def quadratic_bodies(parts):
    """Merge six-node meshes [(nodes, tri6, nv), ...] into one whose first nodes are
    all the triangle corners (body by body), then all the edge nodes.  Returns
    (nodes, tri6, nv, body) with body[T] the index of the part triangle T came from."""
    corners = sum(nv for _, _, nv in parts)
    c_off, e_off = 0, corners
    N, T6, B, C, E = [], [], [], [], []
    for k, (nodes, tri6, nv) in enumerate(parts):
        ne = len(nodes) - nv
        remap = np.concatenate([c_off + np.arange(nv), e_off + np.arange(ne)])
        C.append(nodes[:nv])
        E.append(nodes[nv:])
        T6.append(remap[tri6])
        B.append(np.full(len(tri6), k, np.int32))
        c_off += nv
        e_off += ne
    nodes = np.concatenate(C + E)
    return nodes, np.concatenate(T6).astype(np.int32), corners, np.concatenate(B)


def jitter(X: np.ndarray, tri: np.ndarray, frac: float, seed: int, movable=None) -> np.ndarray:
    """Move each vertex by U(-frac, frac) * (mean length of its edges), per coordinate."""
    rng = np.random.default_rng(seed)
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    L = np.linalg.norm(X[e[:, 0]] - X[e[:, 1]], axis=1)
    s = np.zeros(len(X))
    cnt = np.zeros(len(X))
    np.add.at(s, e[:, 0], L)
    np.add.at(s, e[:, 1], L)
    np.add.at(cnt, e[:, 0], 1)
    np.add.at(cnt, e[:, 1], 1)
    h = s / np.maximum(cnt, 1)
    d = rng.uniform(-frac, frac, size=X.shape) * h[:, None]
    if movable is not None:
        d[~movable] = 0.0
    return X + d


# --------------------------------------------------------------------------- workloads
def sphere_mesh(level: int = 3, V0: float = 1.0, radius: float = 1.0) -> Mesh:
    """Unit-sphere conductor at potential V0 (the single-body Dirichlet case)."""
    X, tri = icosphere(level, radius)
    return Mesh(X, tri, np.zeros(len(tri), np.int32), [{"kind": "conductor", "V0": V0}],
                {"body": "icosphere", "level": level, "radius": radius})


def geodesic_sphere_mesh(freq: int, V0: float = 1.0, jitter_frac: float = 0.0, seed: int = 0) -> Mesh:
    X, tri = geodesic_sphere(freq)
    if jitter_frac > 0:
        X = jitter(X, tri, jitter_frac, seed)
    return Mesh(X, tri, np.zeros(len(tri), np.int32), [{"kind": "conductor", "V0": V0}],
                {"body": "geodesic_sphere", "freq": freq, "jitter": jitter_frac, "seed": seed})


def device_mesh(scale: float = 1.0, seed: int = 2, jitter_frac: float = 0.005,
                eps_r: float = 4.0) -> Mesh:
    """Multi-domain device: conductor sphere (R=1, V0=1) at the origin, floating
    torus (R=2, r=0.3) at z=0 and a dielectric cylinder (radius 0.5, height 2,
    eps_r) centred at (0,0,-3), exterior eps=1.

    Panel counts follow a common target edge length, so that scale=1 gives
    about 20k triangles; the count grows like scale**2.
    """
    m = max(2, int(round(17 * scale)))
    n_v = max(3, int(round(28 * scale)))
    n_u = max(6, int(round(190 * scale)))
    K = max(2, int(round(8 * scale)))
    n_z = max(2, int(round(30 * scale)))
    Xs, Ts = geodesic_sphere(m)
    Xt, Tt = torus(n_u, n_v, 2.0, 0.3, 0.0)
    Xc, Tc = closed_cylinder(0.5, 2.0, (0.0, 0.0, -3.0), K, n_z)
    if jitter_frac > 0:
        Xs = jitter(Xs, Ts, jitter_frac, seed)
        Xt = jitter(Xt, Tt, jitter_frac, seed + 1)
        side = (np.hypot(Xc[:, 0], Xc[:, 1]) > 0.5 - 1e-9) & (np.abs(Xc[:, 2] + 3.0) < 1.0 - 1e-9)
        Xc = jitter(Xc, Tc, jitter_frac, seed + 2, movable=side)
    X, tri, region = _merge([(Xs, Ts, 0), (Xt, Tt, 1), (Xc, Tc, 2)])
    regions = [{"kind": "conductor", "V0": 1.0},
               {"kind": "floating", "floating_id": 0, "eps_plus": 1.0},
               {"kind": "dielectric", "eps_plus": 1.0, "eps_minus": eps_r}]
    info = {"body": "device", "scale": scale, "sphere_freq": m, "torus": (n_u, n_v),
            "cylinder": (K, n_z), "counts": (len(Ts), len(Tt), len(Tc)), "seed": seed,
            "jitter": jitter_frac}
    return Mesh(X, tri, region, regions, info)


def sphere_in_sheet_mesh(level: int, a: float = 1.0, b: float = 2.0, eps_in: float = 4.0,
                         eps_out: float = 1.0, V0: float = 1.0) -> Mesh:
    """Conductor sphere (radius a, potential V0) inside a closed thin floating sheet
    (radius b), with permittivity eps_in between them and eps_out outside: the
    concentric case of Eq. sheets, which has a closed-form solution."""
    X1, T1 = icosphere(level, a)
    X2, T2 = icosphere(level, b)
    X, tri, region = _merge([(X1, T1, 0), (X2, T2, 1)])
    regions = [{"kind": "conductor", "V0": V0},
               {"kind": "sheet", "floating_id": 0, "eps_plus": eps_out, "eps_minus": eps_in}]
    return Mesh(X, tri, region, regions, {"body": "sphere_in_sheet", "level": level, "a": a, "b": b,
                                          "eps_in": eps_in, "eps_out": eps_out})


BUSHING_FOIL_RADII = (0.25, 0.40, 0.55, 0.70, 0.85)
BUSHING_FOIL_LENGTHS = (3.0, 2.6, 2.2, 1.8, 1.4)


def bushing_mesh(scale: float = 1.0, eps_r: float = 4.0, V0: float = 1.0) -> Mesh:
    """Graded-foil bushing analogue (the arrangement of Sec. 5's validation case,
    with made-up dimensions): a high-voltage rod (closed cylinder, radius 0.1,
    length 5, potential V0) inside five coaxial cylindrical foils, open at both
    ends, at the radii BUSHING_FOIL_RADII with the lengths BUSHING_FOIL_LENGTHS
    (centred at z=0).  The outermost foil is grounded (a conductor at 0); the four
    inner ones are thin floating sheets.  All foils lie in one insulator, so both
    sides of a sheet have eps_r.  Edge length about 0.06/scale (about 21k
    triangles at scale 1)."""
    h = 0.06 / scale
    K = max(2, int(round(2.0 * np.pi * 0.1 / h / 6.0)))
    Xr, Tr = closed_cylinder(0.1, 5.0, (0.0, 0.0, 0.0), K, max(2, int(round(5.0 / h))))
    parts = [(Xr, Tr, 0)]
    regions = [{"kind": "conductor", "V0": V0}]
    nf = len(BUSHING_FOIL_RADII)
    for k, (r, L) in enumerate(zip(BUSHING_FOIL_RADII, BUSHING_FOIL_LENGTHS)):
        n_t = max(6, int(round(2.0 * np.pi * r / h)))
        n_z = max(2, int(round(L / h)))
        Xf, Tf = open_cylinder(r, -L / 2.0, L / 2.0, n_t, n_z)
        parts.append((Xf, Tf, len(regions)))
        if k == nf - 1:
            regions.append({"kind": "conductor", "V0": 0.0})
        else:
            regions.append({"kind": "sheet", "floating_id": k, "eps_plus": eps_r, "eps_minus": eps_r})
    X, tri, region = _merge(parts)
    info = {"body": "bushing", "scale": scale, "counts": tuple(len(p[1]) for p in parts), "eps_r": eps_r}
    return Mesh(X, tri, region, regions, info)


def device_family(n: int = 64, n_min: int = 2000, n_max: int = 30000, seed: int = 7,
                  jitter_frac: float = 0.02) -> list:
    """n seeded perturbations of device_mesh for batched runs: triangle counts drawn
    uniformly in [n_min, n_max] (through the scale; counts grow like scale**2 from
    about 20k at scale 1) and every vertex jittered by up to jitter_frac of its mean
    edge length per coordinate."""
    rng = np.random.default_rng(seed)
    target = rng.uniform(n_min, n_max, size=n)
    return [device_mesh(scale=math.sqrt(t / 20068.0), seed=seed * 1000 + 3 * k, jitter_frac=jitter_frac)
            for k, t in enumerate(target)]


# --------------------------------------------------------------------------- points
def ball_points(M: int, rmax: float, rng) -> np.ndarray:
    """M points uniform in the ball |x| < rmax (rejection sampling from the cube)."""
    out = []
    while sum(len(o) for o in out) < M:
        p = rng.uniform(-rmax, rmax, size=(2 * M, 3))
        out.append(p[np.linalg.norm(p, axis=1) < rmax])
    return np.concatenate(out)[:M]


def shell_points(M: int, r0: float, r1: float, rng) -> np.ndarray:
    """M points uniform in volume in the shell r0 < |x| < r1."""
    r = (r0 ** 3 + rng.uniform(0.0, 1.0, M) * (r1 ** 3 - r0 ** 3)) ** (1.0 / 3.0)
    d = rng.normal(size=(M, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return d * r[:, None]


def sphere_eval_points(seed: int = 1, n_in: int = 1000, n_out: int = 1000) -> np.ndarray:
    """n_in points in |x|<0.9 followed by n_out points in 1.5<|x|<3."""
    rng = np.random.default_rng(seed)
    return np.concatenate([ball_points(n_in, 0.9, rng), shell_points(n_out, 1.5, 3.0, rng)])


def device_box_points(M: int, seed: int = 5, half: float = 4.0) -> np.ndarray:
    """M points uniform in [-half, half]^3 outside the device's conductors
    (the sphere |x|<1 and the solid torus); the dielectric's interior is kept."""
    rng = np.random.default_rng(seed)
    out, n = [], 0
    while n < M:
        p = rng.uniform(-half, half, size=(2 * M, 3))
        rho = np.hypot(p[:, 0], p[:, 1])
        in_sphere = np.linalg.norm(p, axis=1) < 1.0
        in_torus = (rho - 2.0) ** 2 + p[:, 2] ** 2 < 0.3 ** 2
        p = p[~(in_sphere | in_torus)]
        out.append(p)
        n += len(p)
    return np.concatenate(out)[:M]


def fibonacci_seeds(L: int, radius: float = 1.0) -> np.ndarray:
    """L Fibonacci points on the sphere |x| = radius: z_k = 1-(2k+1)/L, angle k*pi*(3-sqrt 5)."""
    k = np.arange(L, dtype=np.float64)
    zk = 1.0 - (2.0 * k + 1.0) / L
    ph = k * np.pi * (3.0 - math.sqrt(5.0))
    rxy = np.sqrt(np.maximum(0.0, 1.0 - zk * zk))
    return radius * np.stack([rxy * np.cos(ph), rxy * np.sin(ph), zk], axis=-1)

"""Synthetic inputs (CPU): the seeded device family of the batched workload.

Every mesh must be a closed, consistently oriented surface per body (each edge
shared by exactly two triangles, traversed once in each direction), with triangle
counts in the requested range, reproducible from the seed, and jitter bounded by
the stated fraction of the local edge length.
"""
import numpy as np

from paper_2003_12663_gb300 import meshgen as mg


def _edges_closed_and_oriented(tri):
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    directed = {tuple(x) for x in e}
    assert len(directed) == len(e)                       # no directed edge twice
    return all((b, a) in directed for a, b in directed)  # every edge has its twin


def test_family_counts_seeded_and_closed():
    fam = mg.device_family(5, n_min=2000, n_max=30000, seed=7)
    again = mg.device_family(5, n_min=2000, n_max=30000, seed=7)
    for m, m2 in zip(fam, again):
        assert np.array_equal(m.X, m2.X) and np.array_equal(m.tri, m2.tri)
        assert 1800 <= m.np_ <= 31000
        assert [r["kind"] for r in m.regions] == ["conductor", "floating", "dielectric"]
        for r in range(3):
            assert _edges_closed_and_oriented(m.tri[m.region == r])
    other = mg.device_family(5, seed=8)
    assert any(a.np_ != b.np_ for a, b in zip(fam, other))


def test_family_jitter_bounded():
    base = mg.device_mesh(scale=0.4, seed=3, jitter_frac=0.0)
    jit = mg.device_mesh(scale=0.4, seed=3, jitter_frac=0.02)
    assert np.array_equal(base.tri, jit.tri)
    tri = base.tri
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    L = np.linalg.norm(base.X[e[:, 0]] - base.X[e[:, 1]], axis=1)
    h = np.zeros(len(base.X))
    cnt = np.zeros(len(base.X))
    np.add.at(h, e[:, 0], L)
    np.add.at(h, e[:, 1], L)
    np.add.at(cnt, e[:, 0], 1)
    np.add.at(cnt, e[:, 1], 1)
    h /= cnt
    d = np.abs(jit.X - base.X)
    assert (d <= 0.02 * h[:, None] + 1e-15).all()
    assert d.max() > 0.005 * h.max() * 0.1   # it does move


def test_open_cylinder_sheet():
    """An open cylindrical foil: normals point away from the axis, and its two rims
    are the only boundary (2 n_t edges used by one triangle)."""
    X, tri = mg.open_cylinder(0.5, -1.0, 1.0, 24, 10)
    a, b, c = X[tri[:, 0]], X[tri[:, 1]], X[tri[:, 2]]
    n = np.cross(b - a, c - a)
    ctr = (a + b + c) / 3.0
    assert np.all(n[:, 0] * ctr[:, 0] + n[:, 1] * ctr[:, 1] > 0.0)
    e = np.sort(np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]]), axis=1)
    _, cnt = np.unique(e, axis=0, return_counts=True)
    assert np.sum(cnt == 1) == 2 * 24 and np.all(cnt <= 2)


def test_bushing_and_sheet_meshes():
    m = mg.bushing_mesh(1.0)
    assert 19000 < m.np_ < 23000
    assert m.n_floating == 4
    assert [r["kind"] for r in m.regions] == ["conductor"] + ["sheet"] * 4 + ["conductor"]
    assert m.regions[-1]["V0"] == 0.0
    s = mg.sphere_in_sheet_mesh(2)
    assert s.n_floating == 1 and s.regions[1]["eps_minus"] == 4.0


def test_quadratic_meshes():
    """Six-node triangles: corner nodes first (the P1 unknowns), edge nodes on the
    sphere, every edge node shared by the two triangles of its edge; merging
    bodies keeps all corners ahead of all edge nodes."""
    nodes, tri6, nv = mg.quadratic_sphere(1, 2.0)
    assert nv == 42 and len(nodes) == 42 + 120 and tri6.shape == (80, 6)
    assert np.all(tri6[:, :3] < nv) and np.all(tri6[:, 3:] >= nv)
    assert np.allclose(np.linalg.norm(nodes, axis=1), 2.0)
    _, cnt = np.unique(tri6[:, 3:], return_counts=True)
    assert np.all(cnt == 2)
    n2, t2, nv2 = mg.quadratic_sphere(0, 0.5)
    m, t, nvm, body = mg.quadratic_bodies([(nodes, tri6, nv), (n2 + 3.0, t2, nv2)])
    assert nvm == nv + nv2 and len(m) == len(nodes) + len(n2)
    assert np.all(t[:, :3] < nvm) and np.all(t[:, 3:] >= nvm)
    assert np.allclose(m[t[body == 1]], (n2 + 3.0)[t2])
    assert np.allclose(m[t[body == 0]], nodes[tri6])

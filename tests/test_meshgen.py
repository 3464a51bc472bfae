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

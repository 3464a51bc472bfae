"""bem_adjoint (GPU, through the C ABI) against the oracle's gradient on every
coordinate.

The oracle's gradient (oracle.Problem.adjoint) is a separate, hand-written FP64
reverse pass of the same discrete map: the oracle tracer's steps, the LU solve of
the collocation system, and the pair integrals of the method.  It is pinned on the
CPU by central differences and by the point-charge closed form (test_oracle_adjoint).

* Small meshes with every row kind (conductor, dielectric, closed floating body,
  open sheet with eps+ != eps-): all vertex coordinates, V0 and the permittivities,
  FP64 GPU form, lines traced with h = 0.02.  Both sides differentiate the same
  FP64 computation; they differ by rounding and by the solves (LU against GMRES to
  1e-13), so the tolerance is 1e-6 max(|g|, 1e-3 max|g|) per component.
* The adjoint configuration itself: the 1,280-triangle sphere at V0 = 1 with 256
  Fibonacci lines at h = 1e-3, J = sum of K, all 1,926 vertex coordinates against
  the oracle's gradient stored in tests/golden/adjoint_c3_oracle.txt (written by
  tests/golden/make_adjoint_c3.py, which calls only the oracle).  Same tolerance;
  dJ/dV0 to 1e-8 relative; dJ/deps = 0.
* The mixed form against the oracle to 1e-4 max|g| (FP32 regular pairs).
* Checkpointing: the adjoint recomputes each segment of k steps from a stored
  state; the result does not depend on k (bit for bit), nor on how many lines are
  held at once (to rounding).
"""
import os

import numpy as np
import pytest

from paper_2003_12663_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

H = 0.02
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def bem():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2003_12663_gb300 import bem as B
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return B


def _combine(bodies, regions):
    Xs, Ts, Rs, off = [], [], [], 0
    for (X, tri), r in bodies:
        Xs.append(X)
        Ts.append(tri + off)
        Rs.append(np.full(len(tri), r, np.int32))
        off += len(X)
    return mg.Mesh(np.concatenate(Xs), np.concatenate(Ts).astype(np.int32), np.concatenate(Rs), regions)


def _foil():
    X, T = mg.open_cylinder(0.4, -0.5, 0.5, 12, 4)
    return X + np.array([2.5, 0.0, 0.0]), T


CASES = {
    "sphere": (lambda: mg.sphere_mesh(2), lambda s: s[::4]),
    "dielectric": (lambda: _combine([(mg.icosphere(2, 1.0), 0), (mg.icosphere(2, 0.7, (0.0, 0.0, -2.5)), 1)],
                                    [{"kind": "conductor", "V0": 1.0},
                                     {"kind": "dielectric", "eps_plus": 1.0, "eps_minus": 4.0}]),
                   lambda s: s[s[:, 2] > 0.3][::2]),
    "floating": (lambda: _combine([(mg.icosphere(2, 1.0), 0), (mg.icosphere(2, 0.5, (2.5, 0.3, 0.0)), 1)],
                                  [{"kind": "conductor", "V0": 1.0},
                                   {"kind": "floating", "floating_id": 0, "eps_plus": 1.0}]),
                 lambda s: s[2::5][s[2::5][:, 0] < 0.5]),
    "sheet": (lambda: _combine([(mg.icosphere(2, 1.0), 0), (_foil(), 1)],
                               [{"kind": "conductor", "V0": 1.0},
                                {"kind": "sheet", "floating_id": 0, "eps_plus": 1.0, "eps_minus": 3.0}]),
              lambda s: s[s[:, 0] < -0.2]),
}


def _agree(g, go, rel):
    scale = np.abs(go).max()
    tol = rel * np.maximum(np.abs(go), 1e-3 * scale)
    return np.abs(g - go) <= tol


@pytest.fixture(scope="module", params=list(CASES))
def small(request, oracle_mod):
    make, pick = CASES[request.param]
    mesh = make()
    seeds = pick(mg.fibonacci_seeds(16))
    w = np.random.default_rng(3).uniform(0.5, 1.5, len(seeds))
    P = oracle_mod.Problem(mesh, eta=4.0, g=3)
    u = P.solve()
    ref = P.adjoint(u, seeds, w, oracle_mod.TraceParams(h=H))
    return request.param, mesh, seeds, w, ref


def _gpu_adjoint(bem, mesh, seeds, w, prec, **params):
    ctx = bem.Context(mesh, **params)
    u, _, _ = ctx.solve(prec, tol=1e-13 if prec == bem.FP64 else 1e-10)
    out = ctx.adjoint(u[0], torch.tensor(seeds), torch.tensor(w), prec, h=H)
    ctx.close()
    return [t.cpu().numpy() for t in out]


def test_small_all_coordinates_fp64(bem, small):
    name, mesh, seeds, w, (Ko, gXo, gV0o, gepso) = small
    K, gX, gV0, geps = _gpu_adjoint(bem, mesh, seeds, w, bem.FP64)
    assert np.abs(K - Ko).max() <= 1e-9 * np.abs(Ko).max()
    ok = _agree(gX.reshape(-1), gXo.reshape(-1), 1e-6)
    bad = np.where(~ok)[0]
    assert ok.all(), (name, bad[:10], gX.reshape(-1)[bad[:10]], gXo.reshape(-1)[bad[:10]])
    # derivatives that vanish analytically (eps+ of a closed floating body: its
    # neutrality row is eps+ times a quantity that is 0 at the solution) are rounding
    # noise on both sides; they are compared against the gradient's scale
    scale = max(np.abs(gV0o).max(), np.abs(gXo).max())
    assert np.allclose(gV0, gV0o, rtol=1e-8, atol=1e-12 * scale)
    assert np.allclose(geps, gepso, rtol=1e-6, atol=1e-12 * scale)


def test_small_mixed(bem, small):
    name, mesh, seeds, w, (Ko, gXo, gV0o, gepso) = small
    K, gX, gV0, geps = _gpu_adjoint(bem, mesh, seeds, w, bem.MIXED)
    s = np.abs(gXo).max()
    assert np.abs(gX - gXo).max() <= 1e-4 * s
    assert np.abs(gV0 - gV0o).max() <= 1e-4 * np.abs(gV0o).max()


def test_checkpoint_interval_and_line_chunks(bem):
    """The recomputation from checkpoints is exact: any checkpoint interval gives the
    same bits; holding fewer lines at once only changes the order of the sums."""
    mesh = mg.sphere_mesh(2)
    seeds = mg.fibonacci_seeds(16)[::2]
    w = np.linspace(0.5, 1.5, len(seeds))
    a = _gpu_adjoint(bem, mesh, seeds, w, bem.FP64, adjoint_checkpoint=128, adjoint_lines=16)
    b = _gpu_adjoint(bem, mesh, seeds, w, bem.FP64, adjoint_checkpoint=7, adjoint_lines=16)
    c = _gpu_adjoint(bem, mesh, seeds, w, bem.FP64, adjoint_checkpoint=4096, adjoint_lines=16)
    for x, y, z in zip(a, b, c):
        assert np.array_equal(x, y) and np.array_equal(x, z)
    d = _gpu_adjoint(bem, mesh, seeds, w, bem.FP64, adjoint_lines=3)
    for x, y in zip(a, d):
        assert np.allclose(x, y, rtol=1e-12, atol=1e-15 * np.abs(x).max())


def test_checkpoints_on_split_mesh(bem):
    """On a mesh whose tracer rounds are split over a cluster (9,834 triangles, clusters
    of 3 CTAs), the recomputed segments retrace the forward pass bit for bit: every
    checkpoint interval gives the same gradient, and K is bem_trace_lines' K."""
    mesh = mg.device_mesh(0.7, seed=2)
    seeds = np.array([[0.1, 0.05, 1.0], [-0.2, 0.1, 1.0]])  # above the sphere: lines reach r_max
    seeds = 1.05 * seeds / np.linalg.norm(seeds, axis=1, keepdims=True)
    w = np.array([0.7, 1.3])
    a = _gpu_adjoint(bem, mesh, seeds, w, bem.MIXED, trace_cluster=3, adjoint_checkpoint=128)
    b = _gpu_adjoint(bem, mesh, seeds, w, bem.MIXED, trace_cluster=3, adjoint_checkpoint=7)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    ctx = bem.Context(mesh, trace_cluster=3)
    u, _, _ = ctx.solve(bem.MIXED, tol=1e-10)
    K, st, _, _ = ctx.trace_lines(u[0], torch.tensor(seeds), bem.MIXED, h=H)
    ctx.close()
    assert np.all(st.cpu().numpy() == 1)
    assert np.allclose(a[0], K.cpu().numpy(), rtol=1e-13, atol=0)
    assert np.abs(a[1]).max() > 0


def test_no_workspace(bem):
    mesh = mg.sphere_mesh(1)
    ctx = bem.Context(mesh, adjoint_lines=0)
    u, _, _ = ctx.solve(bem.FP64, tol=1e-12)
    with pytest.raises(bem.BemError) as ei:
        ctx.adjoint(u[0], torch.tensor(mg.fibonacci_seeds(4)), torch.ones(4, dtype=torch.float64), bem.FP64)
    assert ei.value.code == -7
    with pytest.raises(bem.BemError) as ei:
        ctx.matvec_transpose(torch.ones(ctx.nunk, dtype=torch.float64))
    assert ei.value.code == -7
    ctx.close()


def _golden_c3():
    path = os.path.join(HERE, "golden", "adjoint_c3_oracle.txt")
    K, gX = {}, {}
    for line in open(path):
        if line.startswith("#"):
            continue
        p = line.split()
        if p[0] == "J":
            J = float(p[1])
        elif p[0] == "dJ_dV0":
            gV0 = float(p[1])
        elif p[0] == "dJ_deps":
            geps = (float(p[1]), float(p[2]))
        elif p[0] == "K":
            K[int(p[1])] = float(p[2])
        elif p[0] == "gX":
            gX[int(p[1])] = [float(v) for v in p[2:5]]
    return (J, gV0, geps, np.array([K[k] for k in range(len(K))]),
            np.array([gX[v] for v in range(len(gX))]))


def test_config3_all_coordinates(bem):
    """The adjoint configuration: every vertex coordinate of the 1,280-triangle
    sphere, 256 lines, h = 1e-3, against the stored oracle gradient."""
    J_o, gV0_o, geps_o, K_o, gX_o = _golden_c3()
    mesh = mg.sphere_mesh(3)
    seeds = mg.fibonacci_seeds(256)
    ctx = bem.Context(mesh)
    u, _, _ = ctx.solve(bem.FP64, tol=1e-13)
    K, gX, gV0, geps = ctx.adjoint(u[0], torch.tensor(seeds), torch.ones(256, dtype=torch.float64), bem.FP64)
    ctx.close()
    K, gX, gV0, geps = K.cpu().numpy(), gX.cpu().numpy(), gV0.cpu().numpy(), geps.cpu().numpy()
    assert gX.shape == (642, 3) and gX_o.shape == (642, 3)
    assert np.abs(K - K_o).max() <= 1e-9 * np.abs(K_o).max()
    ok = _agree(gX.reshape(-1), gX_o.reshape(-1), 1e-6)
    bad = np.where(~ok)[0]
    assert ok.all(), (bad[:10], gX.reshape(-1)[bad[:10]], gX_o.reshape(-1)[bad[:10]])
    assert abs(gV0[0] - gV0_o) <= 1e-8 * abs(gV0_o)
    assert np.all(geps == 0.0) and geps_o == (0.0, 0.0)
    # per line, the continuum value of dK/dV0 (jump term included) up to the mesh error
    assert abs(gV0_o / 256 - 0.0720913901) < 5e-4

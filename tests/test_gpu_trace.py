"""GPU field-line tracer (bem_trace_lines) against the oracle tracer and the
continuum sphere.

Both tracers run the same integrator on the same sigma; the FP64 form agrees to
rounding (the event roots are solved to 1e-14 h), the mixed form to the FP32 error
of the field (~1e-7) propagated along the line.
"""
import math

import numpy as np
import pytest

from paper_2003_12663_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def K_closed(V0=1.0, c=1e-2, E0=0.5, d=0.1, rmax=10.0):
    rs = math.sqrt(V0 / E0)
    F = lambda r: c * (-V0 * V0 / (3 * r ** 3) + 2 * V0 * E0 / r + E0 * E0 * r)
    return F(rs) - F(1.0) - d * (rmax - rs)


@pytest.fixture(scope="module")
def sphere(oracle_mod):
    import __graft_entry__
    __graft_entry__.build()
    from paper_2003_12663_gb300 import bem
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mesh = mg.sphere_mesh(3)
    ctx = bem.Context(mesh)
    u, _, _ = ctx.solve(bem.FP64, tol=1e-12)
    P = oracle_mod.Problem(mesh, eta=ctx.params.eta, g=ctx.params.far_order)
    yield bem, ctx, u[0], P
    ctx.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_trace_matches_oracle_coarse(sphere, oracle_mod, prec):
    bem, ctx, u, P = sphere
    seeds = mg.fibonacci_seeds(256)[::16]
    K, st, ns, xe = (a.cpu().numpy() for a in ctx.trace_lines(u, torch.tensor(seeds), prec, h=0.01))
    Ko, sto, nso, xeo = P.trace(u.cpu().numpy(), seeds, oracle_mod.TraceParams(h=0.01))
    assert np.array_equal(st, sto) and np.all(st == 1)
    if prec == 0:
        assert np.array_equal(ns, nso)
        assert np.abs(K - Ko).max() < 1e-9 * np.abs(Ko).max()
        assert np.abs(xe - xeo).max() < 1e-9
    else:
        assert np.abs(ns - nso).max() <= 1
        assert np.abs(K - Ko).max() < 1e-5 * np.abs(Ko).max()
        assert np.abs(xe - xeo).max() < 1e-5


def test_trace_config3_full_step(sphere, oracle_mod):
    """256 Fibonacci lines, h = 1e-3: all reach r_max, K near the continuum value,
    four sampled lines equal to the oracle's in FP64."""
    bem, ctx, u, P = sphere
    seeds = mg.fibonacci_seeds(256)
    K, st, ns, xe = (a.cpu().numpy() for a in ctx.trace_lines(u, torch.tensor(seeds), bem.MIXED))
    assert np.all(st == 1)
    assert np.abs(K - K_closed()).max() < 5e-3
    sel = np.array([0, 77, 128, 255])
    K64, st64, ns64, _ = (a.cpu().numpy() for a in ctx.trace_lines(u, torch.tensor(seeds[sel]), bem.FP64))
    Ko, sto, nso, _ = P.trace(u.cpu().numpy(), seeds[sel], oracle_mod.TraceParams(h=1e-3))
    assert np.array_equal(st64, sto) and np.array_equal(ns64, nso)
    assert np.abs(K64 - Ko).max() < 1e-9 * np.abs(Ko).max()
    assert np.abs(K[sel] - Ko).max() < 1e-5 * np.abs(Ko).max()


def test_trace_stop_conditions(sphere, oracle_mod):
    bem, ctx, u, P = sphere
    seeds = mg.fibonacci_seeds(256)[5::50]
    K, st, ns, xe = ctx.trace_lines(u, torch.tensor(seeds), bem.FP64, h=0.01, max_steps=10)
    assert torch.all(st == 3) and torch.all(ns == 10)
    K, st, ns, xe = ctx.trace_lines(u, torch.tensor(seeds), bem.FP64, h=0.01, e_floor=0.25)
    Ko, sto, nso, xeo = P.trace(u.cpu().numpy(), seeds, oracle_mod.TraceParams(h=0.01, e_floor=0.25))
    assert np.array_equal(st.cpu().numpy(), sto) and np.all(sto == 4)
    assert np.array_equal(ns.cpu().numpy(), nso)
    K, st, ns, xe = ctx.trace_lines(u, torch.zeros((0, 3), dtype=torch.float64), bem.FP64)
    assert K.numel() == 0


def test_trace_second_electrode(oracle_mod):
    from paper_2003_12663_gb300 import bem
    X1, T1 = mg.icosphere(2, 1.0)
    X2, T2 = mg.icosphere(2, 0.5, (3.0, 0.0, 0.0))
    mesh = mg.Mesh(np.concatenate([X1, X2]), np.concatenate([T1, T2 + len(X1)]).astype(np.int32),
                   np.concatenate([np.zeros(len(T1), np.int32), np.ones(len(T2), np.int32)]),
                   [{"kind": "conductor", "V0": 1.0}, {"kind": "conductor", "V0": 0.0}])
    ctx = bem.Context(mesh)
    u, _, _ = ctx.solve(bem.FP64, tol=1e-12)
    P = oracle_mod.Problem(mesh, eta=4.0, g=3)
    seeds = np.array([[1.0, 0.013, 0.021], [0.99, 0.1, -0.017], [-1.0, 0.02, 0.03]])
    seeds /= np.linalg.norm(seeds, axis=1, keepdims=True)
    K, st, ns, xe = (a.cpu().numpy() for a in ctx.trace_lines(u[0], torch.tensor(seeds), bem.FP64, h=0.01))
    Ko, sto, nso, xeo = P.trace(u[0].cpu().numpy(), seeds, oracle_mod.TraceParams(h=0.01))
    assert np.array_equal(st, sto) and list(st) == [2, 2, 1]
    assert np.array_equal(ns, nso)
    assert np.abs(K - Ko).max() < 1e-9 and np.abs(xe - xeo).max() < 1e-9
    ctx.close()


@pytest.fixture(scope="module")
def device_split(oracle_mod):
    """The multi-domain device at 9,834 triangles: large enough for the tracer to split
    every round's triangles over the CTAs of a cluster."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_2003_12663_gb300 import bem
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mesh = mg.device_mesh(0.7, seed=2)
    assert mesh.tri.shape[0] >= 8192
    ctx = bem.Context(mesh)
    u, _, _ = ctx.solve(bem.FP64, tol=1e-12)
    ctx.close()
    seeds = mg.fibonacci_seeds(64, radius=1.05)[3::16]
    P = oracle_mod.Problem(mesh, eta=4.0, g=3)
    ref = P.trace(u[0].cpu().numpy(), seeds, oracle_mod.TraceParams(h=0.01))
    return bem, mesh, u[0], seeds, ref


@pytest.mark.parametrize("ncl", [1, 2, 3, 8])
@pytest.mark.parametrize("prec", [0, 1])
def test_trace_cluster_split_matches_oracle(device_split, prec, ncl):
    """Clusters of 1, 2, 3 and 8 CTAs (the triangles of every round split into ncl
    parts, the last of them ragged) trace the oracle's lines: FP64 to rounding with the
    same statuses and step counts, mixed to the FP32 error of the field."""
    bem, mesh, u, seeds, (Ko, sto, nso, xeo) = device_split
    ctx = bem.Context(mesh, trace_cluster=ncl)
    K, st, ns, xe = (a.cpu().numpy() for a in ctx.trace_lines(u, torch.tensor(seeds), prec, h=0.01))
    ctx.close()
    assert np.array_equal(st, sto) and np.all(st > 0)
    if prec == 0:
        assert np.array_equal(ns, nso)
        assert np.abs(K - Ko).max() < 1e-9 * np.abs(Ko).max()
        assert np.abs(xe - xeo).max() < 1e-9
    else:
        assert np.abs(ns - nso).max() <= 1
        assert np.abs(K - Ko).max() < 1e-5 * np.abs(Ko).max()


@pytest.mark.parametrize("prec", [0, 1])
def test_batch_trace_cluster_split_bitwise(device_split, prec):
    """With the same cluster size, the batched tracer gives bem_trace_lines' results bit
    for bit on a split mesh too."""
    bem, mesh, u, seeds, _ = device_split
    ctx = bem.Context(mesh, trace_cluster=4)
    K1, s1, n1, _ = ctx.trace_lines(u, torch.tensor(seeds), prec, h=0.01)
    B = bem.Batch([ctx], nrhs=1)
    K, st, ns = B.trace([u], [seeds], prec, h=0.01)
    assert torch.equal(K[0], K1) and torch.equal(st[0], s1) and torch.equal(ns[0], n1)
    B.close()
    ctx.close()

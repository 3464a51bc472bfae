"""Batched path (bem_batch_*): many uneven meshes x several right-hand sides x many
seeds, through the C ABI, against the FP64 oracle and against the single-mesh calls.

Tolerances (as the single-mesh mixed form):
* products: FP32 regular pairs with compensated sums, so within 2e-6 of the oracle's
  FP64 product (relative to max|y| of the right-hand side);
* solutions after FP64-accurate refinement to 1e-10: sigma within 1e-6 (relative L2)
  of the oracle's LU solution;
* field lines: the batched tracer runs the single-mesh integrator on the same data,
  so K, status and step counts are bit-identical to bem_trace_lines.
"""
import numpy as np
import pytest

from paper_2003_12663_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bem():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2003_12663_gb300 import bem as B
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return B


def _family():
    """Four instances of uneven size and kind: a 20-triangle sphere (one ragged
    tile), a jittered sphere, and two jittered devices (conductor, floating torus,
    dielectric cylinder) of different refinement."""
    return [mg.sphere_mesh(0, V0=1.0),
            mg.geodesic_sphere_mesh(9, V0=1.0, jitter_frac=0.02, seed=4),
            mg.device_mesh(scale=0.3, seed=11, jitter_frac=0.02),
            mg.device_mesh(scale=0.22, seed=12, jitter_frac=0.02)]


@pytest.fixture(scope="module")
def fam(bem, oracle_mod):
    meshes = _family()
    ctxs = [bem.Context(m) for m in meshes]
    probs = [oracle_mod.Problem(m, eta=c.params.eta, g=c.params.far_order) for m, c in zip(meshes, ctxs)]
    mats = [P.assemble() for P in probs]
    yield meshes, ctxs, probs, mats
    for c in ctxs:
        c.close()


def _V0s(meshes, nr):
    """Conductor potentials per right-hand side: V0 in (1, 0.5, -1, 2)."""
    vals = [1.0, 0.5, -1.0, 2.0][:nr]
    out = []
    for m in meshes:
        V = np.zeros((nr, len(m.regions)))
        for r, v in enumerate(vals):
            for k, R in enumerate(m.regions):
                if R["kind"] == "conductor":
                    V[r, k] = v * R["V0"]
        out.append(V)
    return out


def _rhs_oracle(P, V):
    """Oracle right-hand side for conductor potentials V [nregions]."""
    b = np.zeros(P.N + P.F)
    for i in range(P.N):
        R = P.mesh.regions[P.mesh.region[i]]
        if R["kind"] == "conductor":
            b[i] = V[P.mesh.region[i]]
    return b


@pytest.mark.parametrize("nr", [1, 3, 4])
def test_batch_matvec_vs_oracle(fam, bem, nr):
    meshes, ctxs, probs, mats = fam
    rng = np.random.default_rng(100 + nr)
    xs = [rng.standard_normal((nr, c.nunk)) for c in ctxs]
    B = bem.Batch(ctxs, nrhs=nr)
    ys = B.matvec([torch.tensor(x) for x in xs])
    for x, y, A, c in zip(xs, ys, mats, ctxs):
        yg = y.cpu().numpy()
        for r in range(nr):
            ref = A @ x[r]
            err = np.abs(yg[r] - ref).max() / np.abs(ref).max()
            assert err < 2e-6, err
            # the single-mesh mixed product takes the same FP32 decisions
            y1 = c.matvec(torch.tensor(x[r]), bem.MIXED).cpu().numpy()
            assert np.abs(yg[r] - y1).max() / np.abs(y1).max() < 1e-6
    cnt = B.counters()
    assert cnt["far_launches"] == 1
    assert cnt["pairs"] == sum(c.np ** 2 for c in ctxs)
    assert cnt["rhs_pairs"] == nr * cnt["pairs"]
    B.close()


def test_batch_solve_vs_oracle(fam, bem):
    meshes, ctxs, probs, mats = fam
    nr = 4
    V0 = _V0s(meshes, nr)
    B = bem.Batch(ctxs, nrhs=nr)
    us, iters, rel = B.solve([torch.tensor(v) for v in V0], tol=1e-10)
    assert (rel <= 1e-10).all(), rel
    assert (iters > 0).all()
    for k, (u, P, A, V) in enumerate(zip(us, probs, mats, V0)):
        ug = u.cpu().numpy()
        for r in range(nr):
            ref = np.linalg.solve(A, _rhs_oracle(P, V[r]))
            err = np.linalg.norm(ug[r] - ref) / np.linalg.norm(ref)
            assert err < 1e-6, (k, r, err)
    cnt = B.counters()
    assert cnt["graph_launches"] > 0
    assert cnt["far_launches"] >= cnt["graph_launches"]
    assert cnt["arnoldi_steps"] == int(iters.sum())
    B.close()


def test_batch_with_sheets_vs_oracle(bem, oracle_mod):
    """Instances with thin floating sheets (Eq. sheets): the batched product and
    solve against the oracle, four right-hand sides."""
    meshes = [mg.sphere_in_sheet_mesh(2), mg.bushing_mesh(0.25)]
    ctxs = [bem.Context(m) for m in meshes]
    probs = [oracle_mod.Problem(m, eta=c.params.eta, g=c.params.far_order) for m, c in zip(meshes, ctxs)]
    mats = [P.assemble() for P in probs]
    nr = 4
    rng = np.random.default_rng(7)
    xs = [rng.standard_normal((nr, c.nunk)) for c in ctxs]
    B = bem.Batch(ctxs, nrhs=nr)
    ys = B.matvec([torch.tensor(x) for x in xs])
    for x, y, A in zip(xs, ys, mats):
        yg = y.cpu().numpy()
        for r in range(nr):
            ref = A @ x[r]
            assert np.abs(yg[r] - ref).max() / np.abs(ref).max() < 2e-6
    V0 = _V0s(meshes, nr)
    us, iters, rel = B.solve([torch.tensor(v) for v in V0], tol=1e-10)
    assert (rel <= 1e-10).all(), rel
    for k, (u, P, A, V) in enumerate(zip(us, probs, mats, V0)):
        ug = u.cpu().numpy()
        for r in range(nr):
            ref = np.linalg.solve(A, _rhs_oracle(P, V[r]))
            assert np.linalg.norm(ug[r] - ref) / np.linalg.norm(ref) < 1e-6, (k, r)
    B.close()
    for c in ctxs:
        c.close()


def test_batch_solve_matches_single(fam, bem):
    """Per system, the batched solve reaches the single-mesh bem_solve's solution."""
    meshes, ctxs, probs, mats = fam
    B = bem.Batch(ctxs, nrhs=1)
    us, iters, rel = B.solve(None, tol=1e-10)
    for c, u in zip(ctxs, us):
        u1, _, rel1 = c.solve(bem.MIXED, tol=1e-10)
        d = torch.linalg.norm(u[0] - u1[0]) / torch.linalg.norm(u1[0])
        assert d.item() < 1e-8, d.item()
    B.close()


def test_batch_residual_independent(fam, bem):
    """|b - A64 u| / |b| <= tol, with the residual formed by the FP64 single-mesh product."""
    meshes, ctxs, probs, mats = fam
    nr = 2
    V0 = _V0s(meshes, nr)
    B = bem.Batch(ctxs, nrhs=nr)
    us, iters, rel = B.solve([torch.tensor(v) for v in V0], tol=1e-9)
    for c, u, V in zip(ctxs, us, V0):
        b = c.rhs(torch.tensor(V), nrhs=nr)
        for r in range(nr):
            res = b[r] - c.matvec(u[r], bem.FP64)
            assert (torch.linalg.norm(res) / torch.linalg.norm(b[r])).item() <= 1.5e-9
    B.close()


@pytest.mark.parametrize("prec", ["MIXED", "FP64"])
def test_batch_trace_matches_single(fam, bem, prec):
    """One persistent launch over all instances' lines gives bem_trace_lines' results
    bit for bit; an instance may have no lines."""
    meshes, ctxs, probs, mats = fam
    p = getattr(bem, prec)
    B = bem.Batch(ctxs, nrhs=1)
    us, _, _ = B.solve(None, tol=1e-10)
    counts = [3, 0, 5, 4]
    seeds = [mg.fibonacci_seeds(L, radius=1.05) if L else np.zeros((0, 3)) for L in counts]
    tp = dict(h=5e-3, r_max=4.0)
    K, st, ns = B.trace([u[0] for u in us], seeds, p, **tp)
    for c, u, s, Kb, sb, nb in zip(ctxs, us, seeds, K, st, ns):
        if len(s) == 0:
            assert len(Kb) == 0
            continue
        K1, s1, n1, _ = c.trace_lines(u[0], s, p, **tp)
        assert torch.equal(Kb, K1)
        assert torch.equal(sb, s1)
        assert torch.equal(nb, n1)
        assert (s1 > 0).all()
    assert B.counters()["lines"] == sum(counts)
    B.close()


@pytest.mark.parametrize("prec", ["MIXED", "FP64"])
def test_batch_trace_vs_oracle(fam, bem, oracle_mod, prec):
    """Batched lines against the oracle's tracer on the same density: FP64 to
    rounding, mixed within the field tolerance carried along the line (the bounds of
    the single-mesh tracer tests)."""
    meshes, ctxs, probs, mats = fam
    B = bem.Batch(ctxs[:2], nrhs=1)
    us, _, _ = B.solve(None, tol=1e-10)
    seeds = [mg.fibonacci_seeds(4, radius=1.05), mg.fibonacci_seeds(6, radius=1.05)]
    tp = dict(h=5e-3, r_max=4.0)
    K, st, ns = B.trace([u[0] for u in us], seeds, getattr(bem, prec), **tp)
    for P, u, s, Kb, sb, nb in zip(probs[:2], us, seeds, K, st, ns):
        Ko, so, no, _ = P.trace(u[0].cpu().numpy(), s, oracle_mod.TraceParams(**tp))
        Kb, sb, nb = Kb.cpu().numpy(), sb.cpu().numpy(), nb.cpu().numpy()
        assert np.array_equal(sb, so) and np.all(so == 1)
        if prec == "FP64":
            assert np.array_equal(nb, no)
            assert np.abs(Kb - Ko).max() < 1e-9 * np.abs(Ko).max()
        else:
            assert np.abs(nb - no).max() <= 1
            assert np.abs(Kb - Ko).max() < 1e-5 * np.abs(Ko).max()
    B.close()


def test_batch_errors(fam, bem):
    meshes, ctxs, probs, mats = fam
    with pytest.raises(bem.BemError):
        bem.Batch(ctxs, nrhs=5)
    c2 = bem.Context(meshes[0], far_order=5)
    with pytest.raises(bem.BemError):
        bem.Batch([ctxs[0], c2], nrhs=1)   # far_order differs
    c2.close()
    B = bem.Batch(ctxs[:2], nrhs=2)
    with pytest.raises(bem.BemError):
        B.solve(None, tol=1e-8)            # V0 = NULL needs nrhs = 1
    with pytest.raises(bem.BemError):
        B.solve([torch.zeros(2, 1), torch.zeros(2, 1)], tol=1e-8, precision=bem.FP64)
    # zero right-hand sides: nothing to solve, u = 0, relres 0
    us, iters, rel = B.solve([torch.zeros(2, 1), torch.zeros(2, 1)], tol=1e-8)
    assert all(torch.count_nonzero(u).item() == 0 for u in us)
    assert (iters == 0).all() and (rel == 0).all()
    B.close()


def test_batch_device_family_sampled(bem):
    """A sampled batch of the uneven device family (2k-30k triangles, 2% jitter,
    4 right-hand sides): every system converges to 1e-8 by the independent FP64
    residual, and sigma scales with V0 (the systems differ only by the factor)."""
    meshes = mg.device_family(6, seed=7)
    ctxs = [bem.Context(m) for m in meshes]
    V0 = _V0s(meshes, 4)
    B = bem.Batch(ctxs, nrhs=4)
    us, iters, rel = B.solve([torch.tensor(v) for v in V0], tol=1e-8)
    assert (rel <= 1e-8).all()
    for c, u, V in zip(ctxs, us, V0):
        b = c.rhs(torch.tensor(V), nrhs=4)
        for r in range(4):
            res = b[r] - c.matvec(u[r], bem.FP64)
            assert (torch.linalg.norm(res) / torch.linalg.norm(b[r])).item() <= 1.5e-8
        # linearity in V0: u_r / V0_r equals u_0 within the solve tolerance
        for r, s in enumerate([1.0, 0.5, -1.0, 2.0]):
            d = torch.linalg.norm(u[r] / s - u[0]) / torch.linalg.norm(u[0])
            assert d.item() < 2e-5
    B.close()
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("prec,tol", [(1, 1e-5), (0, 1e-11)], ids=["mixed", "fp64"])
def test_batch_eval_field_vs_oracle(fam, bem, prec, tol):
    """bem_batch_eval_field: every instance's points (uneven counts, one instance with
    none, ragged tiles, points 1e-4 off the surface) against the oracle's field, and
    (mixed) against each instance's own bem_eval_field."""
    meshes, ctxs, probs, mats = fam
    B = bem.Batch(ctxs, nrhs=1)
    rng = np.random.default_rng(17)
    us, pts = [], []
    for k, (m, P, A) in enumerate(zip(meshes, probs, mats)):
        us.append(torch.tensor(1.0 + 0.2 * rng.standard_normal(P.N + P.F)))
        if k == 1:
            pts.append(np.zeros((0, 3)))
            continue
        n_box = [300, 0, 1234, 517][k]
        pts.append(np.concatenate([mg.device_box_points(n_box, seed=30 + k),
                                   P.centroids[::23] + 1e-4 * P.normals[::23]]))
    B.reset_counters()
    phi, E = B.eval_field(us, pts, precision=prec)
    torch.cuda.synchronize()
    for k, P in enumerate(probs):
        if len(pts[k]) == 0:
            assert phi[k].numel() == 0
            continue
        pr, Er = P.field(us[k].numpy(), pts[k])
        assert np.abs(phi[k].cpu().numpy() - pr).max() <= tol * np.abs(pr).max()
        assert np.abs(E[k].cpu().numpy() - Er).max() <= tol * np.abs(Er).max()
        if prec == bem.MIXED:
            p1, E1 = ctxs[k].eval_field(us[k], torch.tensor(pts[k]), bem.MIXED)
            assert (E[k] - E1).abs().max().item() <= 1e-5 * E1.abs().max().item()
    if prec == bem.MIXED:
        c = B.counters()
        assert c["eval_pairs"] == sum(len(p) * P.N for p, P in zip(pts, probs))
    B.close()

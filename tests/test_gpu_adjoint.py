"""Adjoint gradient of J = sum_l w_l K_l (bem_adjoint) against central finite
differences (step 1e-5) of the forward solve + trace: the GPU FP64 forward and the
FP64 CPU oracle (LU + oracle tracer).  Tolerance, per component:
|g - g_FD| <= 1e-4 * max(|g_FD|, 1e-3 * max|g_FD|) + 50 ulp(|J|) / step,
the last term being the rounding floor of a difference quotient of J (the forward
is reproducible to a few ulps; below that a finite difference cannot resolve)."""
import numpy as np
import pytest

from paper_2003_12663_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

H = 0.02
STEP = 1e-5


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


def _with(mesh, X=None, regions=None):
    return mg.Mesh(mesh.X if X is None else X, mesh.tri, mesh.region,
                   mesh.regions if regions is None else regions)


def gpu_J(bem, mesh, seeds, w, prec=0):
    ctx = bem.Context(mesh)
    u, _, _ = ctx.solve(prec, tol=1e-13 if prec == 0 else 1e-10)
    K, st, _, _ = ctx.trace_lines(u[0], torch.tensor(seeds), prec, h=H)
    ctx.close()
    assert torch.all(st == 1)
    return float((K.cpu().numpy() * w).sum())


def oracle_J(O, mesh, seeds, w):
    P = O.Problem(mesh, eta=4.0, g=3)
    u = P.solve()
    K, st, _, _ = P.trace(u, seeds, O.TraceParams(h=H))
    assert np.all(st == 1)
    return float((K * w).sum())


def close(g, gfd, J, step=STEP):
    scale = max(np.max(np.abs(gfd)), 1e-30)
    floor = 50 * np.finfo(float).eps * abs(J) / step
    tol = 1e-4 * np.maximum(np.abs(gfd), 1e-3 * scale) + floor
    return np.all(np.abs(g - gfd) <= tol), np.abs(g - gfd) / tol


def run_case(bem, oracle_mod, mesh, seeds, n_coords, n_oracle, fd_regions=()):
    rng = np.random.default_rng(3)
    w = rng.uniform(0.5, 1.5, len(seeds))
    ctx = bem.Context(mesh)
    u, _, _ = ctx.solve(bem.FP64, tol=1e-13)
    K, gX, gV0, geps = ctx.adjoint(u[0], torch.tensor(seeds), torch.tensor(w), bem.FP64, h=H)
    Kt, _, _, _ = ctx.trace_lines(u[0], torch.tensor(seeds), bem.FP64, h=H)
    assert torch.allclose(K, Kt, rtol=0, atol=1e-14)
    J = float((K.cpu().numpy() * w).sum())
    gX, gV0, geps = gX.cpu().numpy(), gV0.cpu().numpy(), geps.cpu().numpy()
    ctx.close()
    # vertex coordinates, FD of the GPU FP64 forward
    flat = rng.choice(mesh.X.size, size=n_coords, replace=False)
    g_fd = []
    for f in flat:
        Xp, Xm = mesh.X.copy(), mesh.X.copy()
        Xp.flat[f] += STEP
        Xm.flat[f] -= STEP
        g_fd.append((gpu_J(bem, _with(mesh, Xp), seeds, w) - gpu_J(bem, _with(mesh, Xm), seeds, w)) / (2 * STEP))
    g_fd = np.array(g_fd)
    ok, err = close(gX.reshape(-1)[flat], g_fd, J)
    assert ok, err
    # the largest few against the oracle's forward
    for f in flat[np.argsort(-np.abs(g_fd))[:n_oracle]]:
        Xp, Xm = mesh.X.copy(), mesh.X.copy()
        Xp.flat[f] += STEP
        Xm.flat[f] -= STEP
        go = (oracle_J(oracle_mod, _with(mesh, Xp), seeds, w) -
              oracle_J(oracle_mod, _with(mesh, Xm), seeds, w)) / (2 * STEP)
        ok, err = close(np.array([gX.reshape(-1)[f]]), np.array([go]), J)
        assert ok, (f, gX.reshape(-1)[f], go)
    # region parameters
    for r, key, col in fd_regions:
        regs_p = [dict(x) for x in mesh.regions]
        regs_m = [dict(x) for x in mesh.regions]
        regs_p[r][key] += STEP
        regs_m[r][key] -= STEP
        gfd = (gpu_J(bem, _with(mesh, regions=regs_p), seeds, w) -
               gpu_J(bem, _with(mesh, regions=regs_m), seeds, w)) / (2 * STEP)
        g = gV0[r] if key == "V0" else geps[r, col]
        ok, err = close(np.array([g]), np.array([gfd]), J)
        assert ok, (r, key, g, gfd)
    return gX, gV0, geps


def test_adjoint_sphere(bem, oracle_mod):
    mesh = mg.sphere_mesh(2)
    seeds = mg.fibonacci_seeds(16)[::4]
    gX, gV0, geps = run_case(bem, oracle_mod, mesh, seeds, 12, 3, [(0, "V0", 0)])
    assert np.all(geps == 0.0)  # no dielectric, no floating body: J does not depend on eps


def test_adjoint_dielectric(bem, oracle_mod):
    """Conductor sphere with a dielectric ball beside it (eps_r = 4); the lines leave
    upward and never cross the interface (|E| jumps across a charged interface, and a
    crossing of E0 located on such a jump has no derivative)."""
    regions = [{"kind": "conductor", "V0": 1.0},
               {"kind": "dielectric", "eps_plus": 1.0, "eps_minus": 4.0}]
    mesh = _combine([(mg.icosphere(2, 1.0), 0), (mg.icosphere(2, 0.7, (0.0, 0.0, -2.5)), 1)], regions)
    seeds = mg.fibonacci_seeds(16)
    seeds = seeds[seeds[:, 2] > 0.3][::2]
    run_case(bem, oracle_mod, mesh, seeds, 10, 2,
             [(0, "V0", 0), (1, "eps_minus", 1), (1, "eps_plus", 0)])


def test_adjoint_floating(bem, oracle_mod):
    regions = [{"kind": "conductor", "V0": 1.0},
               {"kind": "floating", "floating_id": 0, "eps_plus": 1.0}]
    mesh = _combine([(mg.icosphere(2, 1.0), 0), (mg.icosphere(2, 0.5, (2.5, 0.3, 0.0)), 1)], regions)
    seeds = mg.fibonacci_seeds(16)[2::5]
    seeds = seeds[seeds[:, 0] < 0.5]  # lines that do not run into the floating body
    run_case(bem, oracle_mod, mesh, seeds, 10, 2, [(0, "V0", 0)])


def test_adjoint_sheet(bem, oracle_mod):
    """Conductor sphere and an open floating sheet (a short cylindrical foil) beside
    it, with different permittivities on its two sides (Eq. sheets): vertex
    gradients and dJ/d eps+, dJ/d eps- of the sheet against differences.  The
    lines leave away from the foil."""
    regions = [{"kind": "conductor", "V0": 1.0},
               {"kind": "sheet", "floating_id": 0, "eps_plus": 1.0, "eps_minus": 3.0}]
    Xf, Tf = mg.open_cylinder(0.4, -0.5, 0.5, 12, 4)
    mesh = _combine([(mg.icosphere(2, 1.0), 0), ((Xf + np.array([2.5, 0.0, 0.0]), Tf), 1)], regions)
    seeds = mg.fibonacci_seeds(16)
    seeds = seeds[seeds[:, 0] < -0.2]
    gX, gV0, geps = run_case(bem, oracle_mod, mesh, seeds, 10, 2,
                             [(0, "V0", 0), (1, "eps_plus", 0), (1, "eps_minus", 1)])
    assert geps[1, 0] != 0.0 and geps[1, 1] != 0.0


@pytest.mark.slow
def test_adjoint_config3(bem):
    """The configuration the gradient is specified on: 1280-triangle sphere at V0=1,
    256 Fibonacci lines, h = 1e-3.  J = sum of K over every 32nd line (weights 0 on
    the others, so the adjoint still runs all 256); 32 seeded random coordinates
    against central differences of that J; dJ/deps = 0 (no dielectric); dJ/dV0 per
    line near the continuum value 0.0720913901 (jump term included)."""
    mesh = mg.sphere_mesh(3)
    seeds = mg.fibonacci_seeds(256)
    w = np.zeros(len(seeds))
    w[::32] = 1.0
    ctx = bem.Context(mesh)
    u, _, _ = ctx.solve(bem.FP64, tol=1e-13)
    K, gX, gV0, geps = ctx.adjoint(u[0], torch.tensor(seeds), torch.tensor(w), bem.FP64)
    J0 = float((K.cpu().numpy() * w).sum())
    gX = gX.cpu().numpy().reshape(-1)
    ctx.close()
    sub = seeds[::32]

    def J(m):
        c = bem.Context(m)
        uu, _, _ = c.solve(bem.FP64, tol=1e-13)
        Kk, st, _, _ = c.trace_lines(uu[0], torch.tensor(sub), bem.FP64)
        c.close()
        assert torch.all(st == 1)
        return Kk.sum().item()

    flat = np.random.default_rng(3).choice(mesh.X.size, size=32, replace=False)
    gfd = []
    for f in flat:
        Xp, Xm = mesh.X.copy(), mesh.X.copy()
        Xp.flat[f] += STEP
        Xm.flat[f] -= STEP
        gfd.append((J(_with(mesh, Xp)) - J(_with(mesh, Xm))) / (2 * STEP))
    ok, err = close(gX[flat], np.array(gfd), J0)
    assert ok, err
    assert np.all(geps.cpu().numpy() == 0.0)
    assert abs(gV0[0].item() / 8 - 0.0720913901) < 5e-3


def test_adjoint_mixed_close_to_fp64(bem):
    mesh = mg.sphere_mesh(2)
    seeds = mg.fibonacci_seeds(16)[::4]
    w = np.ones(len(seeds))
    ctx = bem.Context(mesh)
    u64, _, _ = ctx.solve(bem.FP64, tol=1e-13)
    _, g64, v64, _ = ctx.adjoint(u64[0], torch.tensor(seeds), torch.tensor(w), bem.FP64, h=H)
    u32, _, _ = ctx.solve(bem.MIXED, tol=1e-10)
    _, g32, v32, _ = ctx.adjoint(u32[0], torch.tensor(seeds), torch.tensor(w), bem.MIXED, h=H)
    ctx.close()
    s = g64.abs().max().item()
    assert (g32 - g64).abs().max().item() < 1e-4 * s
    assert abs(v32[0].item() - v64[0].item()) < 1e-4 * abs(v64[0].item())


def test_autograd_function(bem):
    """torch.autograd through BreakdownK equals bem_adjoint's gradient."""
    from paper_2003_12663_gb300.autograd import BreakdownK
    mesh = mg.sphere_mesh(2)
    seeds = torch.tensor(mg.fibonacci_seeds(16)[::4])
    X = torch.tensor(mesh.X, requires_grad=True)
    V0 = torch.tensor([1.0], dtype=torch.float64, requires_grad=True)
    eps = torch.tensor([[1.0, 1.0]], dtype=torch.float64, requires_grad=True)
    K = BreakdownK.apply(X, V0, eps, mesh, seeds, bem.FP64, {"h": H})
    (K * torch.arange(1, len(K) + 1, dtype=torch.float64, device=K.device)).sum().backward()
    ctx = bem.Context(mesh)
    u, _, _ = ctx.solve(bem.FP64, tol=1e-12)
    w = torch.arange(1, len(K) + 1, dtype=torch.float64)
    _, gX, gV0, _ = ctx.adjoint(u[0], seeds, w, bem.FP64, h=H)
    ctx.close()
    assert torch.allclose(X.grad.cpu(), gX.cpu(), rtol=1e-9, atol=1e-12)
    assert torch.allclose(V0.grad.cpu(), gV0.cpu(), rtol=1e-9)


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-6)])
def test_matvec_transpose(bem, oracle_mod, prec, tol):
    regions = [{"kind": "conductor", "V0": 1.0},
               {"kind": "floating", "floating_id": 0, "eps_plus": 1.0},
               {"kind": "dielectric", "eps_plus": 1.0, "eps_minus": 4.0}]
    mesh = _combine([(mg.icosphere(2, 1.0), 0), (mg.icosphere(2, 0.5, (2.5, 0, 0)), 1),
                     (mg.icosphere(2, 0.7, (0, 0, -2.5)), 2)], regions)
    ctx = bem.Context(mesh)
    P = oracle_mod.Problem(mesh, eta=4.0, g=3)
    A = P.assemble()
    x = np.random.default_rng(5).normal(size=ctx.nunk)
    y = ctx.matvec_transpose(torch.tensor(x), prec).cpu().numpy()
    ref = A.T @ x
    assert np.abs(y - ref).max() / np.abs(ref).max() < tol
    ctx.close()

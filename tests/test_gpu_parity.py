"""GPU (through the C ABI) versus the FP64 CPU oracle, element by element.

Tolerances:
* FP64 form: the same steps as the oracle, so entries, matvecs and fields agree
  to rounding (1e-11 relative to the largest entry of the row / field scale);
  sigma after GMRES to 1e-12 within 1e-9 of the LU solution.
* mixed form: regular pairs in FP32 (unit roundoff 6e-8 per term, compensated
  sums), so entries and matvecs within 2e-6; sigma after FP64 iterative
  refinement within 1e-6 (relative L2), |E| within 1e-5 of the field scale
  max|E| (the target tolerances of the method).
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


MESHES = {
    "sphere_l3": lambda: mg.sphere_mesh(3),
    "device_s03": lambda: mg.device_mesh(scale=0.3),
    # thin floating sheets (Eq. sheets): a closed sheet with a permittivity jump
    # around a conductor sphere, and open foils with a grounded open foil
    "sheet_sphere_l3": lambda: mg.sphere_in_sheet_mesh(3),
    "bushing_s025": lambda: mg.bushing_mesh(0.25),
}


@pytest.fixture(scope="module", params=list(MESHES))
def case(request, bem, oracle_mod):
    mesh = MESHES[request.param]()
    ctx = bem.Context(mesh)
    P = oracle_mod.Problem(mesh, eta=ctx.params.eta, g=ctx.params.far_order)
    A = P.assemble()
    yield request.param, mesh, ctx, P, A
    ctx.close()


def _rel_rows(G, R):
    scale = np.maximum(np.abs(R).max(axis=1, keepdims=True), 1e-300)
    return np.max(np.abs(G - R) / scale)


def test_sizes(case):
    name, mesh, ctx, P, A = case
    assert ctx.np == mesh.np_ and ctx.nunk == mesh.n_unknowns
    assert ctx.near_pairs >= ctx.np  # every row holds at least its own triangle


def test_assemble_rows_fp64(case, bem):
    name, mesh, ctx, P, A = case
    G = ctx.assemble_rows(precision=bem.FP64).cpu().numpy()
    assert _rel_rows(G, A) < 1e-11


def test_assemble_rows_mixed(case, bem):
    name, mesh, ctx, P, A = case
    G = ctx.assemble_rows(precision=bem.MIXED).cpu().numpy()
    assert _rel_rows(G, A) < 2e-6


def test_assemble_row_block(case, bem):
    """A ragged block of rows that includes the neutrality rows, if any."""
    name, mesh, ctx, P, A = case
    r0, r1 = ctx.nunk - 77, ctx.nunk
    G = ctx.assemble_rows(r0, r1, precision=bem.FP64).cpu().numpy()
    assert _rel_rows(G, A[r0:r1]) < 1e-11


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-6), (2, 1e-11)])
def test_matvec(case, bem, prec, tol):
    name, mesh, ctx, P, A = case
    rng = np.random.default_rng(11)
    x = rng.normal(size=(3, ctx.nunk))
    y = ctx.matvec(torch.tensor(x), precision=prec).cpu().numpy()
    ref = x @ A.T
    err = np.abs(y - ref).max(axis=1) / np.abs(ref).max(axis=1)
    assert err.max() < tol, err


@pytest.mark.parametrize("prec", [0, 1])
def test_solve_matches_lu(case, bem, prec):
    name, mesh, ctx, P, A = case
    u_ref = np.linalg.solve(A, P.rhs())
    u, iters, rel = ctx.solve(prec, tol=1e-12)
    u = u[0].cpu().numpy()
    assert rel[0] <= 1e-12
    err = np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref)
    assert err < (1e-9 if prec == 0 else 1e-6), (err, iters)
    # the exact system (closed form for every pair) is within the method's budget
    if name == "sphere_l3":
        from oracle import oracle as O
        u_exact = P.solve(O.EXACT)
        assert np.linalg.norm(u - u_exact) / np.linalg.norm(u_exact) < 1e-6


def test_matvec_df_reproduces_fp64(case, bem):
    """The double-FP32 pass reproduces the FP64 operator, including the pairs the
    FP32 and FP64 classifications disagree on."""
    name, mesh, ctx, P, A = case
    x = torch.tensor(np.random.default_rng(12).normal(size=ctx.nunk))
    y64 = ctx.matvec(x, precision=bem.FP64).cpu().numpy()
    ydf = ctx.matvec(x, precision=bem.DF).cpu().numpy()
    assert np.abs(ydf - y64).max() / np.abs(y64).max() < 1e-12


@pytest.mark.parametrize("nr", [2, 3, 4])
def test_matvec_df_multi_rhs(case, bem, nr):
    """Several right-hand sides in one double-FP32 pass: each equals its own
    single-right-hand-side pass bit for bit, and the oracle's FP64 product to rounding
    (1e-11, the FP64 form's bound)."""
    name, mesh, ctx, P, A = case
    X = np.random.default_rng(40 + nr).normal(size=(nr, ctx.nunk))
    Y = ctx.matvec(torch.tensor(X), precision=bem.DF)
    for r in range(nr):
        y1 = ctx.matvec(torch.tensor(X[r]), precision=bem.DF)
        assert torch.equal(Y[r], y1)
        ref = A @ X[r]
        assert np.abs(Y[r].cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-11


@pytest.mark.parametrize("residual", [0, 1, 2], ids=["df", "fp64", "df_update"])
def test_mixed_solve_residual_modes(case, bem, residual):
    """BEM_MIXED with every refinement residual in double-FP32 or FP64, or (the
    default) the first in double-FP32 and the later ones updated with the mixed product
    of the correction: the FP64 residual of the result meets the tolerance and sigma
    matches LU."""
    name, mesh, ctx, P, A = case
    c2 = bem.Context(mesh, residual=residual)
    u, iters, rel = c2.solve(bem.MIXED, tol=1e-10)
    b = c2.rhs()
    r = (b[0] - c2.matvec(u[0], precision=bem.FP64)).norm() / b[0].norm()
    assert r.item() <= 2e-10, (r.item(), rel)
    u_ref = np.linalg.solve(A, P.rhs())
    uu = u[0].cpu().numpy()
    assert np.linalg.norm(uu - u_ref) / np.linalg.norm(u_ref) < 1e-6
    c2.close()


@pytest.mark.parametrize("prec", [0, 1])
def test_eval_field(case, bem, prec):
    name, mesh, ctx, P, A = case
    u_ref = np.linalg.solve(A, P.rhs())
    if name == "sphere_l3":
        pts = np.concatenate([mg.sphere_eval_points(1, 1000, 1000),
                              # near the surface: 1e-3 and 1e-6 of a panel size off the centroids
                              P.centroids[::7] * (1 + 1e-3), P.centroids[3::11] * (1 - 1e-6)])
    else:
        pts = np.concatenate([mg.device_box_points(1500, 5),
                              P.centroids[::13] + 1e-4 * P.normals[::13]])
    pts = pts[: len(pts) - 5]  # ragged count
    phi_r, E_r = P.field(u_ref, pts)
    phi, E = ctx.eval_field(torch.tensor(u_ref), torch.tensor(pts), precision=prec)
    phi, E = phi.cpu().numpy(), E.cpu().numpy()
    tol = 1e-11 if prec == 0 else 1e-5
    assert np.abs(phi - phi_r).max() / np.abs(phi_r).max() < tol
    assert np.abs(E - E_r).max() / np.abs(E_r).max() < tol


@pytest.mark.parametrize("prec", [0, 1])
def test_surface_field(case, bem, prec):
    name, mesh, ctx, P, A = case
    u_ref = np.linalg.solve(A, P.rhs())
    Es_r = P.surface_field(u_ref)
    Es = ctx.surface_field(torch.tensor(u_ref), precision=prec).cpu().numpy()
    tol = 1e-11 if prec == 0 else 1e-5
    assert np.abs(Es - Es_r).max() / np.abs(Es_r).max() < tol


def test_eval_empty_and_tiny(case, bem):
    name, mesh, ctx, P, A = case
    u = torch.ones(ctx.nunk, dtype=torch.float64)
    phi, E = ctx.eval_field(u, torch.zeros((0, 3), dtype=torch.float64))
    assert phi.numel() == 0 and E.numel() == 0
    pts = np.array([[0.05, -0.02, 7.0]])
    phi, E = ctx.eval_field(u, torch.tensor(pts))
    pr, Er = P.field(np.ones(ctx.nunk), pts)
    assert abs(phi.item() - pr[0]) < 1e-12 * abs(pr[0])


def test_rhs_and_multi_rhs(case, bem):
    name, mesh, ctx, P, A = case
    V0 = np.zeros((2, ctx.nregions))
    for k, r in enumerate(mesh.regions):
        if r["kind"] == "conductor":
            V0[0, k], V0[1, k] = r["V0"], -2.0 * r["V0"]
    b = ctx.rhs(torch.tensor(V0), nrhs=2).cpu().numpy()
    assert np.allclose(b[0], P.rhs()) and np.allclose(b[1], -2.0 * P.rhs())
    u, iters, rel = ctx.solve(0, V0=torch.tensor(V0), tol=1e-11, nrhs=2)
    u = u.cpu().numpy()
    assert np.allclose(u[1], -2.0 * u[0], rtol=1e-8, atol=1e-10 * np.abs(u[0]).max())


# ------------------------------------------------------------ FP32 kernel variants
# The context's tuner picks the FP32 regular-pair kernel (scalar k_far32, packed
# k_far32p with 2 or 4 target pairs per thread) only on meshes of 4,096 triangles or
# more; below that it fixes the 2-pair variant.  Every variant is compared with the
# oracle here, on every mesh above, by fixing it through bem_params.far32_variant.
@pytest.fixture(scope="module", params=[1, 2, 3, 4], ids=lambda v: f"far32v{v}")
def variant_case(request, case, bem):
    name, mesh, ctx, P, A = case
    c = bem.Context(mesh, far32_variant=request.param)
    assert c.counters()["far32_variant"] == request.param
    yield request.param, name, mesh, c, P, A
    c.close()


def test_variant_rows_mixed(variant_case, bem):
    v, name, mesh, ctx, P, A = variant_case
    G = ctx.assemble_rows(precision=bem.MIXED).cpu().numpy()
    assert _rel_rows(G, A) < 2e-6


def test_variant_matvec_mixed(variant_case, bem):
    v, name, mesh, ctx, P, A = variant_case
    x = np.random.default_rng(13).normal(size=(2, ctx.nunk))
    ctx.reset_counters()
    y = ctx.matvec(torch.tensor(x), precision=bem.MIXED).cpu().numpy()
    ref = x @ A.T
    err = np.abs(y - ref).max(axis=1) / np.abs(ref).max(axis=1)
    assert err.max() < 2e-6, err
    c = ctx.counters()
    if v > 1:
        assert c["chunks32p"] > 0   # the packed kernel ran
    else:
        assert c["chunks32p"] == 0  # the scalar kernel ran


def test_variant_eval_field_mixed(variant_case, bem):
    v, name, mesh, ctx, P, A = variant_case
    u_ref = np.linalg.solve(A, P.rhs())
    if name == "sphere_l3":
        pts = np.concatenate([mg.sphere_eval_points(1, 700, 700), P.centroids[::9] * (1 + 1e-4)])
    else:
        pts = np.concatenate([mg.device_box_points(1400, 5), P.centroids[::17] + 1e-4 * P.normals[::17]])
    pts = pts[: len(pts) - 3]
    phi_r, E_r = P.field(u_ref, pts)
    phi, E = ctx.eval_field(torch.tensor(u_ref), torch.tensor(pts), precision=bem.MIXED)
    phi, E = phi.cpu().numpy(), E.cpu().numpy()
    assert np.abs(phi - phi_r).max() / np.abs(phi_r).max() < 1e-5
    assert np.abs(E - E_r).max() / np.abs(E_r).max() < 1e-5


def test_variant_solve_mixed(variant_case, bem):
    v, name, mesh, ctx, P, A = variant_case
    u_ref = np.linalg.solve(A, P.rhs())
    u, iters, rel = ctx.solve(bem.MIXED, tol=1e-10)
    u = u[0].cpu().numpy()
    assert np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref) < 1e-6

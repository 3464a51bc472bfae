"""The regular-pair kernels at the size the benchmark step runs them: the
multi-domain device with 20,068 triangles (conductor sphere, floating torus with
its neutrality row, dielectric cylinder), against the oracle.

* Full matrix-free products, all 20,069 rows, for every FP32 kernel variant
  (scalar k_far32; packed k_far32p with 2 and 4 target pairs per thread), the
  FP64 form and the double-FP32 residual form.  The oracle's reference is its own
  matrix-free product (direct summation at every centroid, then the row equations
  of Eqs. Final1-Final4), 4e8 pair integrals.
* The field at 2,000 points: a tight cluster above the sphere (so that whole
  target tiles sit far from most triangle chunks) and uniform box points.
* Blocks of 256 dense rows across the boundaries of two bodies.

At this size the packed kernel meets all three of its paths: chunks summed without
classification ("fast"), masked chunks, and phi-only tiles of conductor rows;
the counters show each was taken.  Tolerances as in test_gpu_parity.py: FP64 1e-11
of the largest entry, mixed 2e-6 for products and rows, 1e-5 of max|E| for fields.
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


@pytest.fixture(scope="module")
def dev20k(oracle_mod):
    mesh = mg.device_mesh(scale=1.0, seed=2)
    assert mesh.np_ == 20068
    P = oracle_mod.Problem(mesh, eta=4.0, g=3)
    rng = np.random.default_rng(2020)
    # a smooth positive density with noise, and one floating potential
    x = 1.0 + 0.1 * rng.standard_normal(mesh.n_unknowns)
    y_ref = P.matvec(x)
    c = np.array([0.0, 0.0, 1.6])
    d = rng.standard_normal((1024, 3))
    d *= (0.3 * rng.random(1024) ** (1 / 3) / np.linalg.norm(d, axis=1))[:, None]
    pts = np.concatenate([c + d, mg.device_box_points(976, seed=55)])
    phi_r, E_r = P.field(x, pts)
    return mesh, P, x, y_ref, pts, phi_r, E_r


def _rel(y, ref):
    return np.abs(y - ref).max() / np.abs(ref).max()


@pytest.mark.parametrize("variant", [1, 2, 3, 4], ids=lambda v: f"far32v{v}")
def test_product_and_field_per_variant(bem, dev20k, variant):
    mesh, P, x, y_ref, pts, phi_r, E_r = dev20k
    ctx = bem.Context(mesh, far32_variant=variant)
    try:
        ctx.reset_counters()
        y = ctx.matvec(torch.tensor(x), precision=bem.MIXED).cpu().numpy()
        assert _rel(y, y_ref) < 2e-6
        c = ctx.counters()
        if variant > 1:
            assert 0 < c["fast_chunks32p"] < c["chunks32p"], c   # both chunk paths taken
            assert c["phi_pairs"][bem.MIXED] > 0, c               # phi-only conductor tiles
        else:
            assert c["chunks32p"] == 0
        ctx.reset_counters()
        phi, E = ctx.eval_field(torch.tensor(x), torch.tensor(pts), precision=bem.MIXED)
        assert _rel(phi.cpu().numpy(), phi_r) < 1e-5
        assert _rel(E.cpu().numpy(), E_r) < 1e-5
        if variant > 1:
            c = ctx.counters()
            assert c["fast_chunks32p"] > 0, c                     # the clustered tile
        assert ctx.counters()["far32_variant"] == variant
    finally:
        ctx.close()


@pytest.fixture(scope="module")
def ctx20k(bem, dev20k):
    mesh = dev20k[0]
    ctx = bem.Context(mesh)
    yield ctx
    ctx.close()


@pytest.mark.parametrize("prec", [0, 2], ids=["fp64", "df"])
def test_product_fp64_forms(bem, dev20k, ctx20k, prec):
    mesh, P, x, y_ref, pts, phi_r, E_r = dev20k
    y = ctx20k.matvec(torch.tensor(x), precision=prec).cpu().numpy()
    assert _rel(y, y_ref) < 1e-11


def test_field_fp64(bem, dev20k, ctx20k):
    mesh, P, x, y_ref, pts, phi_r, E_r = dev20k
    phi, E = ctx20k.eval_field(torch.tensor(x), torch.tensor(pts), precision=bem.FP64)
    assert _rel(phi.cpu().numpy(), phi_r) < 1e-11
    assert _rel(E.cpu().numpy(), E_r) < 1e-11


def test_tuned_context_matches(bem, dev20k, ctx20k):
    """The context as the benchmark creates it (variant picked by timing)."""
    mesh, P, x, y_ref, pts, phi_r, E_r = dev20k
    assert ctx20k.counters()["far32_variant"] in (1, 2, 3, 4)
    y = ctx20k.matvec(torch.tensor(x), precision=bem.MIXED).cpu().numpy()
    assert _rel(y, y_ref) < 2e-6


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-6)], ids=["fp64", "mixed"])
@pytest.mark.parametrize("body", ["sphere|torus", "torus|cylinder"])
def test_row_block(bem, dev20k, ctx20k, prec, tol, body):
    """256 consecutive rows across the boundary of two bodies (conductor and
    floating rows, or floating and dielectric rows) against rows built from the
    oracle's pair integrals."""
    mesh, P, x, y_ref, pts, phi_r, E_r = dev20k
    N, F = P.N, P.F
    n_s, n_t, n_c = mesh.info["counts"]
    r0 = (n_s if body == "sphere|torus" else n_s + n_t) - 128
    r1 = r0 + 256
    idx = np.arange(r0, r1)
    S, G = P.pair_block(P.centroids[r0:r1], idx)
    Kp = np.einsum("ijk,ik->ij", G, P.normals[r0:r1])
    ref = np.zeros((256, N + F))
    for ii, i in enumerate(idx):
        R = mesh.regions[mesh.region[i]]
        if R["kind"] == "conductor":
            ref[ii, :N] = S[ii]
        elif R["kind"] == "floating":
            ref[ii, :N] = S[ii]
            ref[ii, N + R["floating_id"]] = -1.0
        else:
            ep, em = R["eps_plus"], R["eps_minus"]
            ref[ii, :N] = (ep - em) * Kp[ii]
            ref[ii, i] += 0.5 * (ep + em)
    A = ctx20k.assemble_rows(r0, r1, precision=prec).cpu().numpy()
    scale = np.abs(ref).max(axis=1, keepdims=True)
    assert np.max(np.abs(A - ref) / scale) < tol


def test_refinement_residual_update(bem, dev20k):
    """The default refinement forms one double-FP32 residual per solve and updates the
    later ones with the mixed product of the correction: on the 20k device the true
    residual of the result (FP64 product) still meets the tolerance, and the solution
    is the every-step double-FP32 one to 1e-6."""
    mesh = dev20k[0]
    out = {}
    for mode in (bem.RESIDUAL_DF_UPDATE, bem.RESIDUAL_DF):
        ctx = bem.Context(mesh, residual=mode)
        ctx.reset_counters()
        u, iters, rel = ctx.solve(bem.MIXED, tol=1e-8)
        c = ctx.counters()
        b = ctx.rhs()[0]
        r = (b - ctx.matvec(u[0], precision=bem.FP64)).norm() / b.norm()
        out[mode] = (u[0].cpu().numpy(), r.item(), rel[0], c["matvecs"][bem.DF])
        ctx.close()
    uu, ru, relu, ndf_u = out[bem.RESIDUAL_DF_UPDATE]
    ud, rd, reld, ndf_d = out[bem.RESIDUAL_DF]
    assert ru <= 1.05e-8 and abs(ru - relu) <= 5e-10, (ru, relu)
    assert rd <= 1.05e-8
    assert ndf_u == 1 and ndf_d >= 2, (ndf_u, ndf_d)
    assert np.linalg.norm(uu - ud) / np.linalg.norm(ud) < 1e-6


@pytest.fixture(scope="module")
def many_points(oracle_mod, dev20k):
    """12,288 points in random order (uniform box points, a tight cluster and points
    1e-4 off the surface), with the oracle's field: chunks this large are evaluated in
    spatial order by the packed kernel."""
    mesh, P, x = dev20k[0], dev20k[1], dev20k[2]
    rng = np.random.default_rng(77)
    pts = np.concatenate([mg.device_box_points(10240, seed=56), dev20k[4][:1024],
                          P.centroids[::20][:1024] + 1e-4 * P.normals[::20][:1024]])
    pts = pts[rng.permutation(len(pts))]
    phi_r, E_r = P.field(x, pts)
    return pts, phi_r, E_r


@pytest.mark.parametrize("variant", [2, 3, 4], ids=lambda v: f"far32v{v}")
def test_field_in_spatial_order(bem, dev20k, many_points, variant):
    """bem_eval_field sorts each chunk of at least 4,096 points by cell of a 16^3 grid
    along the Morton curve before the packed kernel: the field matches the oracle
    (1e-5 of max|phi|, max|E|), several times more triangle chunks are then summed
    unmasked than in input order (at this density, 2.5 box points per cell, a tenth or
    more of them), and the result is the unordered evaluation's (chunks of 4,095
    points) to FP32 rounding."""
    x = dev20k[2]
    pts, phi_r, E_r = many_points
    ctx = bem.Context(dev20k[0], far32_variant=variant)
    ctx.reset_counters()
    phi, E = ctx.eval_field(torch.tensor(x), torch.tensor(pts), precision=bem.MIXED)
    c = ctx.counters()
    ctx.close()
    phi, E = phi.cpu().numpy(), E.cpu().numpy()
    assert _rel(phi, phi_r) < 1e-5
    assert _rel(E, E_r) < 1e-5
    assert c["fast_chunks32p"] > 0.1 * c["chunks32p"], c
    small = bem.Context(dev20k[0], far32_variant=variant, max_points=4095)
    small.reset_counters()
    phi2, E2 = small.eval_field(torch.tensor(x), torch.tensor(pts), precision=bem.MIXED)
    c2 = small.counters()
    small.close()
    assert 4 * c2["fast_chunks32p"] < c["fast_chunks32p"], (c, c2)
    assert _rel(phi2.cpu().numpy(), phi) < 2e-6
    assert _rel(E2.cpu().numpy(), E) < 2e-6

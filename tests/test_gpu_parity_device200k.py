"""The benchmark step's workload at its full size, in the launch configuration the
benchmark times: the multi-domain device at 199,920 triangles (conductor sphere,
floating torus, dielectric cylinder), its context created with the default
parameters (kernel shape picked by the tuner), and 1e6 box points evaluated in
chunks of 131,072 (each put in Morton cell order for the packed kernel).

The oracle cannot form these products (4e10 pair integrals each), so sampled outputs
are compared, each of which the oracle computes on its own:
* 48 rows of the mixed and of the FP64 matrix-free product (conductor, floating and
  dielectric rows; the neutrality rows need every row and are left out): the
  oracle's direct summation at those centroids, then the row equations of Eqs.
  Final1-Final3;
* phi and E at 200 of the 1e6 points.
Tolerances as in test_gpu_parity.py: FP64 1e-11 and mixed 2e-6 of the largest
sampled row value, 1e-5 of the largest sampled |phi| and |E| for the field.
"""
import numpy as np
import pytest

from paper_2003_12663_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SCALE = (200000 / 20068.0) ** 0.5


@pytest.fixture(scope="module")
def bem():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2003_12663_gb300 import bem as B
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return B


@pytest.fixture(scope="module")
def dev200k(bem, oracle_mod):
    mesh = mg.device_mesh(scale=SCALE, seed=2)
    assert mesh.np_ == 199920
    P = oracle_mod.Problem(mesh, eta=4.0, g=3)
    ctx = bem.Context(mesh)
    rng = np.random.default_rng(200)
    x = 1.0 + 0.1 * rng.standard_normal(mesh.n_unknowns)
    yield mesh, P, ctx, x, rng
    ctx.close()


def _oracle_rows(mesh, P, x, rows):
    """y_i of Eqs. Final1-Final3 at the given (non-neutrality) rows, from the oracle's
    phi and E at those centroids (own panel: the principal value)."""
    N = mesh.np_
    phi, E = P.field(x, P.centroids[rows], rows)
    y = np.empty(len(rows))
    for k, i in enumerate(rows):
        R = mesh.regions[mesh.region[i]]
        if R["kind"] == "conductor":
            y[k] = phi[k]
        elif R["kind"] == "floating":
            y[k] = phi[k] - x[N + R["floating_id"]]
        else:
            ep, em = R["eps_plus"], R["eps_minus"]
            y[k] = 0.5 * (ep + em) * x[i] + (ep - em) * (E[k] @ P.normals[i])
    return y


def test_sampled_product_rows(bem, dev200k):
    mesh, P, ctx, x, rng = dev200k
    kinds = np.array([mesh.regions[r]["kind"] for r in mesh.region])
    rows = np.sort(np.concatenate([rng.choice(np.where(kinds == k)[0], 16, replace=False)
                                   for k in ("conductor", "floating", "dielectric")]))
    ref = _oracle_rows(mesh, P, x, rows)
    scale = np.abs(ref).max()
    ctx.reset_counters()
    ym = ctx.matvec(torch.tensor(x), precision=bem.MIXED).cpu().numpy()
    c = ctx.counters()
    assert c["far32_variant"] >= 2 and 0 < c["fast_chunks32p"] < c["chunks32p"], c
    assert np.abs(ym[rows] - ref).max() <= 2e-6 * scale
    y64 = ctx.matvec(torch.tensor(x), precision=bem.FP64).cpu().numpy()
    assert np.abs(y64[rows] - ref).max() <= 1e-11 * scale


def test_sampled_field_of_a_million_points(bem, dev200k):
    mesh, P, ctx, x, rng = dev200k
    pts = mg.device_box_points(1000000, seed=5)
    phi, E = ctx.eval_field(torch.tensor(x), torch.tensor(pts, device="cuda"), bem.MIXED)
    sel = np.sort(rng.choice(len(pts), 200, replace=False))
    phi_r, E_r = P.field(x, pts[sel])
    phi, E = phi.cpu().numpy()[sel], E.cpu().numpy()[sel]
    assert np.abs(phi - phi_r).max() <= 1e-5 * np.abs(phi_r).max()
    assert np.abs(E - E_r).max() <= 1e-5 * np.abs(E_r).max()

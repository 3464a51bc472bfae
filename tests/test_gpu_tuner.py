"""The tuner of the FP32 regular-pair kernel's shape (bem_create): on a mesh of 4,096
triangles or more every candidate (variant 1, 2, 3, 4 x CTA slots per SM 2, 4, 8) is timed
on the mesh's own mixed matvec and the fastest is kept; the choice goes into a
process-wide table keyed by device, size bucket and far_order, from which later
contexts take it.  Whatever the choice, the product is the same to the FP32 bound."""
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


def test_tuner_times_candidates_then_uses_table(bem):
    bem.clear_tuning_table()
    mesh = mg.device_mesh(scale=0.5, seed=2)
    assert mesh.np_ >= 4096
    c1 = bem.Context(mesh)
    t1 = c1.tuning()
    assert t1["source"] == "timed" and len(t1["candidates"]) == 12
    best = min(t1["candidates"], key=lambda d: d["ms"])
    assert (t1["far32_variant"], t1["far32_slots"]) == (best["variant"], best["slots"])
    assert all(d["ms"] > 0 for d in t1["candidates"])
    # a second mesh of the same size bucket: taken from the table, no timing
    c2 = bem.Context(mg.device_mesh(scale=0.5, seed=3, jitter_frac=0.01))
    t2 = c2.tuning()
    assert t2["source"] == "table" and t2["bucket"] == t1["bucket"]
    assert (t2["far32_variant"], t2["far32_slots"]) == (t1["far32_variant"], t1["far32_slots"])
    # fixed variant and small meshes are not timed
    c3 = bem.Context(mesh, far32_variant=1)
    assert c3.tuning()["source"] == "fixed" and c3.tuning()["far32_variant"] == 1
    c4 = bem.Context(mg.sphere_mesh(2))
    assert c4.tuning()["source"] == "fixed"
    # the product does not depend on the shape beyond FP32 rounding
    x = torch.tensor(np.random.default_rng(4).normal(size=c1.nunk))
    y1 = c1.matvec(x, bem.MIXED)
    y3 = c3.matvec(x, bem.MIXED)
    y64 = c1.matvec(x, bem.FP64)
    s = y64.abs().max().item()
    assert (y1 - y64).abs().max().item() < 2e-6 * s
    assert (y3 - y64).abs().max().item() < 2e-6 * s
    for c in (c1, c2, c3, c4):
        c.close()

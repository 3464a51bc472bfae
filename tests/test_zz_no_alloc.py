"""bem_eval_field_static: the allocation-free variant of the field evaluation.

It exists for callers that cannot allocate device memory when they evaluate the
field (their GPU memory belongs to their own arena after start-up).  Its scratch
is one fixed array in the library's static device memory, shared by all calls on a
device.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2003_12663_gb300 import meshgen as mg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def setup():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2003_12663_gb300 import bem
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    mesh = mg.device_mesh(scale=0.3)
    ctx = bem.Context(mesh)
    u, _, _ = ctx.solve(bem.FP64, tol=1e-10)
    yield bem, ctx, u[0]
    ctx.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 1e-5)])
def test_static_scratch_matches_eval_field(setup, prec, tol):
    """Two calls in a row (different point sets, so the second call runs on
    whatever the first left in the shared array) agree with bem_eval_field."""
    bem, ctx, u = setup
    for seed, M in ((5, 3001), (6, 777)):
        pts = torch.tensor(mg.device_box_points(M, seed=seed))
        phi_r, E_r = ctx.eval_field(u, pts, prec)
        phi, E = ctx.eval_field_static(u, pts, prec)
        torch.cuda.synchronize()
        scale_p = phi_r.abs().max().item()
        scale_E = E_r.abs().max().item()
        assert (phi - phi_r).abs().max().item() <= tol * scale_p
        assert (E - E_r).abs().max().item() <= tol * scale_E


def test_static_scratch_limits(setup):
    bem, ctx, u = setup
    pts = torch.zeros((65537, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(bem.BemError) as ei:
        ctx.eval_field_static(u, pts)
    assert ei.value.code == -7 and "65536" in str(ei.value)
    phi, E = ctx.eval_field_static(u, torch.zeros((0, 3), dtype=torch.float64))
    assert phi.numel() == 0


def test_static_call_allocates_nothing(setup):
    """With phi and E passed in, a call changes neither torch's allocator nor the
    device's free memory (after a first call, which may load the kernels' module)."""
    bem, ctx, u = setup
    pts = torch.tensor(mg.device_box_points(4096, seed=8), device="cuda")
    phi = torch.empty(4096, dtype=torch.float64, device="cuda")
    E = torch.empty((4096, 3), dtype=torch.float64, device="cuda")
    ctx.eval_field_static(u, pts, bem.MIXED, phi=phi, E=E)
    torch.cuda.synchronize()
    a0 = torch.cuda.memory_allocated()
    f0, _ = torch.cuda.mem_get_info()
    for prec in (bem.MIXED, bem.FP64):
        ctx.eval_field_static(u, pts, prec, phi=phi, E=E)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == a0
    f1, _ = torch.cuda.mem_get_info()
    assert f1 == f0

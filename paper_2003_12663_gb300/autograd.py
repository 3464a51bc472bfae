"""torch.autograd wrapper: the breakdown integral K_l (Eq. Breakdowncrit) of every
field line as a differentiable function of the vertex coordinates, the region
potentials V0 and the permittivities.

Forward: bem_create (mesh with the given vertices and region data) -> bem_solve ->
bem_trace_lines.  Backward: bem_adjoint with dL/dK = grad_output.  Argument
marshalling only; both directions run in libbem.so.
"""
from __future__ import annotations

import numpy as np
import torch

from . import bem
from .meshgen import Mesh


def _regions_with(regions, V0, eps):
    out = []
    for r, R in enumerate(regions):
        R = dict(R)
        if R["kind"] == "conductor":
            R["V0"] = float(V0[r])
        if R["kind"] in ("floating", "dielectric", "sheet"):
            R["eps_plus"] = float(eps[r, 0])
        if R["kind"] in ("dielectric", "sheet"):
            R["eps_minus"] = float(eps[r, 1])
        out.append(R)
    return out


class BreakdownK(torch.autograd.Function):
    """K = BreakdownK.apply(X, V0, eps, mesh, seeds, precision, trace_params)

    X: (nv, 3) float64 vertex coordinates; V0: (nregions,) potentials of conductor
    regions (other entries unused); eps: (nregions, 2) (eps_plus, eps_minus);
    mesh: meshgen.Mesh giving triangles and region kinds; seeds: (L, 3).
    Returns K: (L,) on the GPU."""

    @staticmethod
    def forward(ctx, X, V0, eps, mesh, seeds, precision=bem.FP64, trace_params=None):
        tp = dict(trace_params or {})
        Xn = X.detach().cpu().numpy().astype(np.float64)
        regions = _regions_with(mesh.regions, V0.detach().cpu().numpy(), eps.detach().cpu().numpy())
        m = Mesh(Xn, mesh.tri, mesh.region, regions)
        c = bem.Context(m)
        u, _, _ = c.solve(precision, tol=1e-12 if precision == bem.FP64 else 1e-10)
        K, st, _, _ = c.trace_lines(u[0], seeds, precision, **tp)
        ctx.c, ctx.u, ctx.seeds, ctx.precision, ctx.tp = c, u[0], seeds, precision, tp
        ctx.dev = X.device
        return K.to(X.device)

    @staticmethod
    def backward(ctx, gK):
        w = gK.detach().to(device="cuda", dtype=torch.float64).contiguous()
        _, gX, gV0, geps = ctx.c.adjoint(ctx.u, ctx.seeds, w, ctx.precision, **ctx.tp)
        ctx.c.close()
        return gX.to(ctx.dev), gV0.to(ctx.dev), geps.to(ctx.dev), None, None, None, None

"""Pins of the oracle's field-line tracer (Eq. Breakdowncrit: K = int alpha_eff(|E|) ds).

Closed form: a unit sphere at potential V0 has E = V0 x/|x|^3 outside, so a radial
line from r=1 to r_max=10 crosses |E| = E0 at r* = sqrt(V0/E0) and
  K(V0) = int_1^{r*} c (V0/r^2 - E0)^2 dr - d (r_max - r*),
  dK/dV0 = 2c int_1^{r*} (V0/r^2 - E0)/r^2 dr + d / (2 sqrt(V0 E0))
(the last term comes from the jump of alpha_eff at the moving crossing point; it is
only reproduced if the integrator locates that crossing).
"""
import math

import numpy as np
import pytest

from paper_2003_12663_gb300 import meshgen as mg

C, E0, D, RMAX = 1e-2, 0.5, 0.1, 10.0


def K_closed(V0):
    rs = math.sqrt(V0 / E0)
    F = lambda r: C * (-V0 * V0 / (3 * r ** 3) + 2 * V0 * E0 / r + E0 * E0 * r)
    return F(rs) - F(1.0) - D * (RMAX - rs)


def dK_closed(V0):
    rs = math.sqrt(V0 / E0)
    G = lambda r: 2 * C * (-V0 / (3 * r ** 3) + E0 / r)
    return G(rs) - G(1.0) + D / (2 * math.sqrt(V0 * E0))


def test_closed_form_values():
    # the numbers quoted for this configuration (c=1e-2, E0=0.5, d=0.1, V0=1)
    assert K_closed(1.0) == pytest.approx(-0.858317220, abs=2e-9)
    assert dK_closed(1.0) == pytest.approx(0.0720913901, abs=2e-10)
    h = 1e-6
    assert dK_closed(1.0) == pytest.approx((K_closed(1 + h) - K_closed(1 - h)) / (2 * h), rel=1e-7)


def test_point_charge_lines_converge_at_fourth_order(oracle_mod):
    seeds = mg.fibonacci_seeds(7)
    errs = []
    for h in (0.04, 0.02, 0.01):
        K, st, ns, xe = oracle_mod.trace_point_charge(seeds, 1.0, oracle_mod.TraceParams(h=h))
        assert np.all(st == 1)
        assert np.allclose(np.linalg.norm(xe, axis=1), RMAX, atol=1e-10)
        errs.append(np.max(np.abs(K - K_closed(1.0))))
    assert errs[-1] < 1e-9
    assert errs[0] / errs[1] > 10 and errs[1] / errs[2] > 10, errs


def test_event_location_gives_the_jump_derivative(oracle_mod):
    """Central differences in V0 (step 1e-6) reproduce dK/dV0 including the
    jump term d / (2 sqrt(V0 E0))."""
    seeds = mg.fibonacci_seeds(3)
    tp = oracle_mod.TraceParams(h=1e-2)
    s = 1e-6
    Kp, *_ = oracle_mod.trace_point_charge(seeds, 1.0 + s, tp)
    Km, *_ = oracle_mod.trace_point_charge(seeds, 1.0 - s, tp)
    assert np.allclose((Kp - Km) / (2 * s), dK_closed(1.0), rtol=2e-6)


def test_stop_conditions(oracle_mod):
    seeds = mg.fibonacci_seeds(4)
    # step limit
    K, st, ns, xe = oracle_mod.trace_point_charge(seeds, 1.0, oracle_mod.TraceParams(h=0.01, max_steps=10))
    assert np.all(st == 3) and np.all(ns == 10)
    assert np.allclose(np.linalg.norm(xe, axis=1), 1.1, atol=1e-12)
    # field floor, checked at step starts
    K, st, ns, xe = oracle_mod.trace_point_charge(seeds, 1.0, oracle_mod.TraceParams(h=0.01, e_floor=0.25))
    assert np.all(st == 4)
    assert np.all(np.abs(np.linalg.norm(xe, axis=1) - 2.0) <= 0.01 + 1e-12)
    # field lines of a negative potential run the other way round but still outward
    K, st, ns, xe = oracle_mod.trace_point_charge(seeds, -1.0, oracle_mod.TraceParams(h=0.02))
    assert np.all(st == 1)
    assert np.allclose(K, K_closed(1.0), atol=1e-6)


@pytest.mark.slow
def test_bem_sphere_lines_approach_continuum(oracle_mod):
    """Field of the discrete solution on the 1280-triangle sphere: K within the
    discretisation error of the continuum value."""
    P = oracle_mod.Problem(mg.sphere_mesh(3), eta=4.0, g=3)
    u = P.solve()
    seeds = mg.fibonacci_seeds(256)[::32]
    K, st, ns, xe = P.trace(u, seeds, oracle_mod.TraceParams(h=0.01))
    assert np.all(st == 1)
    assert np.max(np.abs(K - K_closed(1.0))) < 5e-3


@pytest.mark.slow
def test_line_hits_second_electrode(oracle_mod):
    """A line from a sphere at V0=1 toward a grounded sphere stops on the grounded
    sphere's surface (status 2)."""
    X1, T1 = mg.icosphere(2, 1.0)
    X2, T2 = mg.icosphere(2, 0.5, (3.0, 0.0, 0.0))
    mesh = mg.Mesh(np.concatenate([X1, X2]), np.concatenate([T1, T2 + len(X1)]).astype(np.int32),
                   np.concatenate([np.zeros(len(T1), np.int32), np.ones(len(T2), np.int32)]),
                   [{"kind": "conductor", "V0": 1.0}, {"kind": "conductor", "V0": 0.0}])
    P = oracle_mod.Problem(mesh, eta=4.0, g=3)
    u = P.solve()
    # seeds off the mesh vertices (the flat-triangle field is singular on edges/vertices)
    seeds = np.array([[1.0, 0.013, 0.021], [0.99, 0.1, -0.017]])
    seeds /= np.linalg.norm(seeds, axis=1, keepdims=True)
    K, st, ns, xe = P.trace(u, seeds, oracle_mod.TraceParams(h=0.01))
    assert np.all(st == 2), st
    r2 = np.linalg.norm(xe - [3.0, 0.0, 0.0], axis=1)
    assert np.all((r2 > 0.45) & (r2 <= 0.5 + 1e-9)), r2
    # a seed on a vertex meets the singular field and stops with status -1
    K, st, ns, xe = P.trace(u, np.array([[1.0, 0.0, 0.0]]), oracle_mod.TraceParams(h=0.01))
    assert st[0] == -1 and ns[0] == 0

"""Pins of the oracle's thin floating sheets (Eq. sheets): a floating conductor
modelled by one surface, whose neutrality row takes the displacement field of
both sides, int (eps+ + eps-)/2 sigma + (eps+ - eps-) K'sigma dS = 0.

Units: phi = int sigma / (4 pi r) dS; sigma is the total (free + bound) charge
density that the single layer carries, i.e. the jump of E.n across the surface.
"""
import numpy as np
import pytest

from paper_2003_12663_gb300 import meshgen as mg


def sheet_closed_form(a, b, eps_in, eps_out, V0):
    """Conductor sphere (radius a, potential V0) inside a closed floating sheet of
    radius b; eps_in between them, eps_out outside.  The sheet carries no free
    charge, so the displacement field is D = q/r^2 (q = Q_free / 4 pi) for r > a and
    E = D/eps.  Integrating E from infinity:
      V_b = q / (eps_out b),   V0 = V_b + q (1/a - 1/b) / eps_in.
    The single layer's densities are the jumps of E.n:
      sigma_a = q / (eps_in a^2),   sigma_b = q (1/eps_out - 1/eps_in) / b^2.
    Returns (V_b, sigma_a, sigma_b)."""
    q = V0 / (1.0 / (eps_out * b) + (1.0 / a - 1.0 / b) / eps_in)
    return q / (eps_out * b), q / (eps_in * a * a), q * (1.0 / eps_out - 1.0 / eps_in) / (b * b)


def test_closed_form_values():
    """The closed form at (a, b, eps_in, eps_out) = (1, 2, 4, 1): q = 1.6; and the
    homogeneous case, where the sheet sits at the potential a/b of the point charge
    and carries nothing."""
    Vb, sa, sb = sheet_closed_form(1.0, 2.0, 4.0, 1.0, 1.0)
    assert (Vb, sa, sb) == pytest.approx((0.8, 0.4, 0.3), rel=1e-15)
    Vb, sa, sb = sheet_closed_form(1.0, 2.0, 1.0, 1.0, 1.0)
    assert (Vb, sa, sb) == pytest.approx((0.5, 1.0, 0.0), rel=1e-15, abs=1e-15)


def _errors(O, level, a, b, eps_in, eps_out):
    mesh = mg.sphere_in_sheet_mesh(level, a, b, eps_in, eps_out)
    P = O.Problem(mesh, eta=4.0, g=3)
    u = P.solve()
    Vb, sa, sb = sheet_closed_form(a, b, eps_in, eps_out, 1.0)
    area = P.area
    ua, ub = u[: P.N][mesh.region == 0], u[: P.N][mesh.region == 1]
    Aa, Ab = area[mesh.region == 0], area[mesh.region == 1]
    # area-weighted L2 errors of sigma, relative to the conductor's density
    ea = np.sqrt(np.sum(Aa * (ua - sa) ** 2) / np.sum(Aa)) / sa
    eb = np.sqrt(np.sum(Ab * (ub - sb) ** 2) / np.sum(Ab)) / sa
    return np.array([abs(u[P.N] - Vb) / Vb, ea, eb]), P, u, mesh


@pytest.mark.slow
def test_sheet_around_sphere_with_permittivity_jump(oracle_mod):
    """eps- = 4 inside the sheet, eps+ = 1 outside: the sheet's potential and both
    densities approach the closed form.  The (eps+ - eps-) K' term makes the rate
    first order: K' on a flat panel misses the curvature of the own panel (its
    principal value is 0), as for a dielectric interface.  The free charge of the
    sheet, sum_i A_i (eps+ E+.n - eps- E-.n) from the field just off its centroids,
    is zero: this fixes the sides and signs of Eq. sheets."""
    e2, _, _, _ = _errors(oracle_mod, 2, 1.0, 2.0, 4.0, 1.0)
    e3, P, u, mesh = _errors(oracle_mod, 3, 1.0, 2.0, 4.0, 1.0)
    assert np.all(e3 < [1.2e-2, 5e-2, 2.5e-2]), e3
    assert np.all(e2 / e3 > 1.5), (e2, e3)
    sel = np.where(mesh.region == 1)[0]
    c, n, A = P.centroids[sel], P.normals[sel], P.area[sel]
    _, Ep = P.field(u, c + 1e-7 * n)
    _, Em = P.field(u, c - 1e-7 * n)
    Dp = 1.0 * np.einsum("ij,ij->i", Ep, n)
    Dm = 4.0 * np.einsum("ij,ij->i", Em, n)
    assert abs(np.sum(A * (Dp - Dm))) < 1e-5 * np.sum(A * np.abs(Dp))
    # with the permittivities swapped in the row the free charge would not vanish
    assert abs(np.sum(A * (4.0 * np.einsum("ij,ij->i", Ep, n) - np.einsum("ij,ij->i", Em, n)))) > \
        1e-2 * np.sum(A * np.abs(Dp))


def test_sheet_in_homogeneous_medium(oracle_mod):
    """eps+ = eps-: the neutrality row is the sheet's total charge, which the solve
    makes zero; the sheet floats at a/b (at O(h^2), no K' term is left) and carries
    almost nothing."""
    e2, _, _, _ = _errors(oracle_mod, 2, 1.0, 2.0, 1.0, 1.0)
    e3, P, u, mesh = _errors(oracle_mod, 3, 1.0, 2.0, 1.0, 1.0)
    assert np.all(e3 < [1e-3, 6e-3, 3e-3]), e3
    assert e2[0] / e3[0] > 3.5, (e2, e3)
    q_sheet = np.sum((u[: P.N] * P.area)[mesh.region == 1])
    q_cond = np.sum((u[: P.N] * P.area)[mesh.region == 0])
    assert abs(q_sheet) < 1e-12 * abs(q_cond)


def test_sheet_without_inner_field_is_a_floating_conductor(oracle_mod):
    """A closed sheet with eps- = 0 (no displacement field on its inside, as in a
    conductor's interior) gives the equation of a floating conductor (Eq.
    constraint): the same matrix up to rounding."""
    X1, T1 = mg.icosphere(2, 1.0)
    X2, T2 = mg.icosphere(2, 0.5, (2.5, 0.0, 0.0))

    def mesh(reg2):
        return mg.Mesh(np.concatenate([X1, X2]), np.concatenate([T1, T2 + len(X1)]).astype(np.int32),
                       np.concatenate([np.zeros(len(T1), np.int32), np.ones(len(T2), np.int32)]),
                       [{"kind": "conductor", "V0": 1.0}, reg2])

    Af = oracle_mod.Problem(mesh({"kind": "floating", "floating_id": 0, "eps_plus": 2.0})).assemble()
    As = oracle_mod.Problem(mesh({"kind": "sheet", "floating_id": 0, "eps_plus": 2.0,
                                  "eps_minus": 0.0})).assemble()
    assert np.allclose(As, Af, rtol=1e-14, atol=1e-15 * np.abs(Af).max())
    assert not np.allclose(
        oracle_mod.Problem(mesh({"kind": "sheet", "floating_id": 0, "eps_plus": 2.0,
                                 "eps_minus": 1.0})).assemble(), Af)


@pytest.mark.slow
def test_bushing_analogue_foil_potentials(oracle_mod):
    """Rod at 1, grounded outer foil, four floating foils between them in one
    insulator: each floating foil carries zero net charge, and by the maximum
    principle its potential lies strictly between 0 and 1; nested foils grade it
    down outward."""
    mesh = mg.bushing_mesh(0.25)
    P = oracle_mod.Problem(mesh, eta=4.0, g=3)
    u = P.solve()
    V = u[P.N:]
    assert len(V) == 4
    assert np.all((V > 0.0) & (V < 1.0)), V
    assert np.all(np.diff(V) < 0.0), V
    q = u[: P.N] * P.area
    q_rod = abs(np.sum(q[mesh.region == 0]))
    for f in range(4):
        assert abs(np.sum(q[mesh.region == f + 1])) < 1e-12 * q_rod

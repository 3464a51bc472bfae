"""Pins of the oracle's single-pair integrals against things other than itself.

* textbook closed forms (the in-plane potential of an equilateral triangle),
* scipy's adaptive 2-D quadrature (an independent brute force),
* the solid-angle theorem on closed meshes,
* the jump of the normal field across a charged sheet (Eq. ADL / Jump),
* the far-field (monopole) limit,
* polynomial exactness of the Duffy/Gauss rule,
* convergence of the paper's subdivision scheme (Sec. 4) to the closed form.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_2003_12663_gb300 import meshgen as mg

FOUR_PI = 4.0 * math.pi


def _brute(x, a, b, c):
    """S and G of a flat triangle by scipy.dblquad in an orthonormal in-plane frame."""
    e1 = (b - a) / np.linalg.norm(b - a)
    nrm = np.cross(b - a, c - a)
    nrm /= np.linalg.norm(nrm)
    e2 = np.cross(nrm, e1)
    # triangle in the frame: (0,0), (Lb,0), (cx,cy), cy > 0
    Lb = np.linalg.norm(b - a)
    cx, cy = np.dot(c - a, e1), np.dot(c - a, e2)

    def y_of(s, t):
        return a + s * e1 + t * e2

    def lo(t):
        return t * cx / cy

    def hi(t):
        return Lb + t * (cx - Lb) / cy

    def integ(f):
        v, err = integrate.dblquad(lambda s, t: f(y_of(s, t)), 0.0, cy, lo, hi,
                                   epsabs=1e-14, epsrel=1e-13)
        return v

    S = integ(lambda y: 1.0 / np.linalg.norm(x - y)) / FOUR_PI
    G = np.array([integ(lambda y, k=k: (x - y)[k] / np.linalg.norm(x - y) ** 3) for k in range(3)])
    return S, G / FOUR_PI


def test_equilateral_self_potential(oracle_mod):
    """In-plane potential at the centroid of an equilateral triangle of side L:
    int 1/r dS = 3 edges x inradius x 2 asinh(sqrt 3) = sqrt(3) L ln(2+sqrt 3)."""
    for L in (1.0, 0.037, 5.0):
        a = np.array([0.3, -0.2, 0.7])
        b = a + L * np.array([1.0, 0.0, 0.0])
        c = a + L * np.array([0.5, math.sqrt(3) / 2, 0.0])
        x = (a + b + c) / 3.0
        S, G = oracle_mod.tri_exact(x, a, b, c, True)
        assert S * FOUR_PI == pytest.approx(math.sqrt(3) * L * math.log(2 + math.sqrt(3)), rel=1e-13)
        # symmetric: the in-plane field at the centroid vanishes, PV normal part is 0
        assert np.max(np.abs(G)) < 1e-13


@pytest.mark.parametrize("case", range(6))
def test_closed_form_vs_adaptive_quadrature(oracle_mod, case):
    rng = np.random.default_rng(100 + case)
    a, b, c = rng.normal(size=(3, 3))
    if np.dot(np.cross(b - a, c - a), [0, 0, 1]) < 0:
        b, c = c, b
    ctr = (a + b + c) / 3
    nrm = np.cross(b - a, c - a)
    nrm /= np.linalg.norm(nrm)
    scale = np.linalg.norm(b - a)
    targets = {
        "far": ctr + 3.0 * scale * rng.normal(size=3),
        "above": ctr + 0.05 * scale * nrm + 0.1 * scale * (b - a),
        "below": ctr - 0.02 * scale * nrm,
        "in_plane_out": a + 1.3 * (b - a) + 0.2 * (c - a),   # outside, in the plane
        "over_edge": 0.5 * (a + b) + 0.01 * scale * nrm,
    }
    for name, x in targets.items():
        S, G = oracle_mod.tri_exact(x, a, b, c)
        Sb, Gb = _brute(x, a, b, c)
        assert S == pytest.approx(Sb, rel=1e-9, abs=1e-13), name
        assert np.allclose(G, Gb, rtol=1e-8, atol=1e-10 * np.linalg.norm(Gb)), name


def test_solid_angle_closed_surfaces(oracle_mod):
    """-4 pi G_j(x).n_j is the solid angle of panel j; over a closed surface the
    sum is 4 pi for x inside and 0 outside (Gauss)."""
    bodies = [mg.icosphere(2), mg.torus(24, 8), mg.closed_cylinder(0.5, 2.0, (0, 0, -3), 3, 5)]
    inside = [np.array([0.1, -0.2, 0.3]), np.array([2.05, 0.0, 0.1]), np.array([0.1, 0.2, -3.5])]
    outside = [np.array([1.5, 0.0, 0.2]), np.array([0.0, 0.0, 0.0]), np.array([0.0, 0.7, -3.0])]
    for (X, tri), xin, xout in zip(bodies, inside, outside):
        geom = oracle_mod.panel_geometry(X, tri)
        for x, want in ((xin, FOUR_PI), (xout, 0.0)):
            tot = 0.0
            for j, t in enumerate(tri):
                _, G = oracle_mod.tri_exact(x, X[t[0]], X[t[1]], X[t[2]])
                tot += -FOUR_PI * np.dot(G, geom[j, 0:3])
            assert tot == pytest.approx(want, abs=1e-11)


def test_normal_jump_and_principal_value(oracle_mod):
    """Eq. (ADL)/(Jump): across a sheet of unit density the normal field jumps by
    1 (in units where phi = int sigma/(4 pi r)); the in-plane part is continuous
    and the principal value is the mean of the two sides."""
    rng = np.random.default_rng(7)
    a, b, c = rng.normal(size=(3, 3))
    nrm = np.cross(b - a, c - a)
    nrm /= np.linalg.norm(nrm)
    x0 = 0.2 * a + 0.5 * b + 0.3 * c
    for d in (1e-6, 1e-9):
        _, Gp = oracle_mod.tri_exact(x0 + d * nrm, a, b, c)
        _, Gm = oracle_mod.tri_exact(x0 - d * nrm, a, b, c)
        assert np.dot(Gp - Gm, nrm) == pytest.approx(1.0, abs=1e3 * d)
        # the normal field is odd in the height, the in-plane part even
        assert abs(np.dot(Gp + Gm, nrm)) < 1e-12
        assert np.allclose(Gp - np.dot(Gp, nrm) * nrm, Gm - np.dot(Gm, nrm) * nrm, atol=1e3 * d)
    ctr = (a + b + c) / 3
    _, Gpv = oracle_mod.tri_exact(ctr, a, b, c, True)
    _, Gp = oracle_mod.tri_exact(ctr + 1e-9 * nrm, a, b, c)
    _, Gm = oracle_mod.tri_exact(ctr - 1e-9 * nrm, a, b, c)
    assert abs(np.dot(Gpv, nrm)) < 1e-15
    assert np.allclose(Gpv, 0.5 * (Gp + Gm), atol=1e-7)


def test_monopole_limit(oracle_mod):
    """S -> A/(4 pi |x-c|) with relative error O((R/D)^2): the first moment of a
    triangle about its centroid vanishes."""
    a, b, c = np.array([0.0, 0, 0]), np.array([1.0, 0.1, 0]), np.array([0.3, 0.9, 0.2])
    ctr = (a + b + c) / 3
    A = 0.5 * np.linalg.norm(np.cross(b - a, c - a))
    d = np.array([0.3, -0.5, 0.8])
    d /= np.linalg.norm(d)
    errs = []
    for D in (4.0, 8.0, 16.0, 32.0):
        S, G = oracle_mod.tri_exact(ctr + D * d, a, b, c)
        errs.append(abs(S * FOUR_PI * D / A - 1.0))
        assert np.allclose(G * FOUR_PI * D * D / A, d, atol=5.0 / D ** 2)
    ratios = [errs[i] / errs[i + 1] for i in range(3)]
    assert all(3.0 < r < 5.0 for r in ratios), ratios


@pytest.mark.parametrize("g", [1, 2, 3, 4, 5])
def test_far_rule_polynomial_exactness(oracle_mod, g):
    """The Duffy/Gauss rule with g points per direction integrates every
    monomial s^p t^q of degree p+q <= 2g-1 over the reference triangle
    (0,0),(1,0),(0,1) exactly: int s^p t^q = p! q! / (p+q+2)!."""
    u, wu, v, wv = oracle_mod.far_rule(g)
    # Duffy map with vertex order a=(0,0), b=(1,0), c=(0,1): y = a + u(b-a) + u v (c-b)
    for p in range(2 * g):
        for q in range(2 * g - p):
            tot = 0.0
            for uk, wk in zip(u, wu):
                for vl, wl in zip(v, wv):
                    s, t = uk * (1 - vl), uk * vl
                    tot += 2 * 0.5 * uk * wk * wl * s ** p * t ** q
            exact = math.factorial(p) * math.factorial(q) / math.factorial(p + q + 2)
            assert tot == pytest.approx(exact, rel=1e-12, abs=1e-15)


def test_far_rule_converges_to_closed_form(oracle_mod):
    """The C-side Duffy map: for a far target every rule order agrees with the
    closed form, and the error drops fast with the order."""
    a, b, c = np.array([0.0, 0, 0]), np.array([1.0, 0.1, 0]), np.array([0.3, 0.9, 0.2])
    x = np.array([0.4, 0.3, 2.5])
    S0, G0 = oracle_mod.tri_exact(x, a, b, c)
    errs = []
    for g in (1, 2, 3, 4, 6, 8):
        S, G = oracle_mod.tri_quad(x, a, b, c, oracle_mod.far_rule(g))
        errs.append(max(abs(S - S0) / S0, np.linalg.norm(G - G0) / np.linalg.norm(G0)))
    assert errs[-1] < 1e-13
    assert all(errs[i + 1] < errs[i] for i in range(4))


def test_subdivision_scheme_converges_to_closed_form(oracle_mod):
    """Sec. 4 near-singular scheme (closest point, split, Duffy) -> closed form."""
    a, b, c = np.array([0.0, 0, 0]), np.array([1.0, 0, 0]), np.array([0.5, math.sqrt(3) / 2, 0])
    for x in (np.array([0.3, 0.2, 0.01]), np.array([0.5, -0.01, 0.002]), np.array([1.2, 0.0, 0.03])):
        S0, G0 = oracle_mod.tri_exact(x, a, b, c)
        S, G = oracle_mod.tri_subdivide(x, a, b, c, 48)
        assert S == pytest.approx(S0, rel=1e-10)
        assert np.allclose(G, G0, rtol=1e-8, atol=1e-10)
    # singular pair: collocation point on the triangle, potential only
    x = np.array([0.4, 0.25, 0.0])
    S0, _ = oracle_mod.tri_exact(x, a, b, c)
    S, _ = oracle_mod.tri_subdivide(x, a, b, c, 32)
    assert S == pytest.approx(S0, rel=1e-11)


def test_classification_threshold(oracle_mod):
    """Sec. 4: a pair is regular iff D > eta R (strict); regular pairs take the
    Duffy/Gauss rule, the others the closed form."""
    X = np.array([[0.0, 0, 0], [1.0, 0, 0], [0.0, 1.0, 0]])
    tri = np.array([[0, 1, 2]], np.int32)
    mesh = mg.Mesh(X, tri, np.zeros(1, np.int32), [{"kind": "conductor", "V0": 1.0}])
    P = oracle_mod.Problem(mesh, eta=2.0, g=2)
    cc, R = P.geom[0, 7:10], P.geom[0, 10]
    d = np.array([0.0, 0.6, 0.8])
    for k, want_quad in ((0.999999, False), (1.000001, True)):
        x = cc + k * 2.0 * R * d
        S, G = P.pair_block(x[None, :])
        Sq, _ = oracle_mod.tri_quad(x, *X, P.rule)
        Se, _ = oracle_mod.tri_exact(x, *X)
        assert abs(Sq - Se) > 1e-6
        assert S[0, 0] == (Sq if want_quad else Se)

"""Pins of the oracle for the paper's own discretisation (mapped linear basis on
curved quadratic triangles, vertex collocation; Sec. 3, Sec. 4, Eq. Matrix):

* on flat triangles the three basis integrals add up to the closed-form integral of
  a constant density (regular, near-singular and singular pairs);
* from a vertex of a flat triangle the integral has a closed form, and the vertex's
  own basis function carries exactly half of it;
* on curved triangles every pair type matches scipy's adaptive quadrature;
* the quadratic sphere's area and the conductor sphere's density converge at
  fourth order (the flat P0 discretisation converges at first or second);
* the quadrature parameters do not change the solution.
"""
import math

import numpy as np
import pytest

from paper_2003_12663_gb300 import meshgen as mg

FOUR_PI = 4.0 * math.pi


@pytest.fixture(scope="module")
def C():
    from oracle import p1curved
    return p1curved


def _shaped_triangles(n, seed):
    """Well-shaped flat triangles: an equilateral triangle with every corner moved
    by up to 20 % of its side, rotated, scaled and shifted at random."""
    rng = np.random.default_rng(seed)
    base = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.5, math.sqrt(3.0) / 2.0, 0.0]])
    out = []
    for _ in range(n):
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        P = (base + rng.uniform(-0.2, 0.2, size=(3, 3))) @ Q.T * rng.uniform(0.5, 2.0) + rng.normal(size=3)
        out.append(P)
    return out


def _flat6(a, b, c):
    return np.array([a, b, c, (a + b) / 2, (b + c) / 2, (c + a) / 2])


def test_flat_reduction_to_closed_form(C, oracle_mod):
    """sum_k int lambda_k / (4 pi r) = int 1 / (4 pi r) (the closed form) for targets
    far away, at 2R (regular), just above and below the surface, next to an edge
    and a corner, and in the plane outside (near-singular).  The regular rule is
    at its worst at D = 2R straight above the triangle (~1e-12)."""
    worst = {"regular": 0.0, "near": 0.0}
    for a, b, c in _shaped_triangles(6, 11):
        P6 = _flat6(a, b, c)
        cc, R = C.circumcircle(a, b, c)
        n = np.cross(b - a, c - a)
        n /= np.linalg.norm(n)
        ctr = (a + b + c) / 3.0
        cases = [(cc + 2.0001 * R * n, "regular"), (cc + 10.0 * R * np.array([0.6, 0.0, 0.8]), "regular"),
                 (ctr + 0.1 * R * n, "near"), (ctr - 1e-6 * R * n, "near"),
                 (0.5 * (a + b) + 0.01 * R * n, "near"), (b - 1e-4 * R * n, "near"),
                 (a + 0.2 * (a - ctr), "near"), (0.3 * a + 0.7 * c + 0.05 * R * n, "near")]
        for x, kind in cases:
            S, _ = oracle_mod.tri_exact(x, a, b, c)
            v = C.pair_integrals(x, P6, kind)
            worst[kind] = max(worst[kind], abs(v.sum() - S) / abs(S))
    assert worst["regular"] < 5e-12 and worst["near"] < 1e-13, worst


def test_vertex_closed_form_and_half(C):
    """From vertex A of a flat triangle, in polar coordinates about A:
    int 1/r dS = int rho(theta) dtheta = d (asinh tan phi2 - asinh tan phi1), with
    d the distance from A to the opposite edge and phi the angles of its ends seen
    from the foot of the perpendicular.  The basis function of A, 1 - rho/rho(theta)
    along each ray, integrates to exactly half of that."""
    for a, b, c in _shaped_triangles(4, 12):
        P6 = _flat6(a, b, c)
        X = [a, b, c]
        for k in range(3):
            A, B, Cc = X[k], X[(k + 1) % 3], X[(k + 2) % 3]
            e = (Cc - B) / np.linalg.norm(Cc - B)
            foot = B + np.dot(A - B, e) * e
            d = np.linalg.norm(A - foot)
            closed = d * (np.arcsinh(np.dot(Cc - foot, e) / d) - np.arcsinh(np.dot(B - foot, e) / d)) / FOUR_PI
            v = C.pair_integrals(A, P6, "singular", corner=k)
            assert v.sum() == pytest.approx(closed, rel=1e-13)
            assert v[k] == pytest.approx(0.5 * closed, rel=1e-13)


def test_equilateral_vertex_value(C):
    """Side 1: from a vertex, int 1/r dS = (sqrt(3)/2) ln 3 (phi = +-30 degrees)."""
    a, b, c = np.array([0.0, 0, 0]), np.array([1.0, 0, 0]), np.array([0.5, math.sqrt(3) / 2, 0])
    v = C.pair_integrals(a, _flat6(a, b, c), "singular", corner=0)
    assert v.sum() * FOUR_PI == pytest.approx(math.sqrt(3) / 2 * math.log(3.0), rel=1e-14)
    assert v[1] == pytest.approx(v[2], rel=1e-13)  # symmetry


@pytest.mark.slow
def test_curved_triangle_against_adaptive_quadrature(C):
    """A curved triangle of the quadratic sphere: the near-singular (a neighbouring
    vertex, points 0.05 off the surface) and singular (own corner) integrals of each
    basis function against scipy's adaptive dblquad over the reference triangle."""
    integrate = pytest.importorskip("scipy.integrate")
    nodes, tri6, nv = mg.quadratic_sphere(1)
    T = 5
    P6 = nodes[tri6[T]]

    def ref(x):
        out = []
        for k in range(3):
            def f(eta, xi):
                y, J = C.surface(P6, np.array([xi]), np.array([eta]))
                return C.linear(np.array([xi]), np.array([eta]))[0, k] * J[0] / np.linalg.norm(x - y[0])
            v, _ = integrate.dblquad(f, 0, 1, 0, lambda xi: 1 - xi, epsabs=1e-14, epsrel=1e-12)
            out.append(v / FOUR_PI)
        return np.array(out)

    yc, _ = C.surface(P6, np.array([1 / 3]), np.array([1 / 3]))
    yc = yc[0]
    nrm = yc / np.linalg.norm(yc)
    others = [v for v in range(nv) if v not in tri6[T, :3]]
    xn = nodes[others[int(np.argmin([np.linalg.norm(nodes[v] - yc) for v in others]))]]
    for x in (xn, yc + 0.05 * nrm, yc - 0.05 * nrm):
        r = ref(x)
        assert np.abs(C.pair_integrals(x, P6, "near") - r).max() < 1e-12 * np.abs(r).max()
    x = nodes[tri6[T, 1]]
    r = ref(x)
    assert np.abs(C.pair_integrals(x, P6, "singular", corner=1) - r).max() < 1e-12 * np.abs(r).max()


def test_quadratic_sphere_area_fourth_order(C):
    """The curved triangles' area tends to 4 pi at O(h^4) (error falls ~16x per
    level); the flat triangles' area at O(h^2)."""
    errs, flat = [], []
    for level in (1, 2):
        nodes, tri6, nv = mg.quadratic_sphere(level)
        errs.append(abs(C.CurvedProblem(nodes, tri6, nv).integrate() - FOUR_PI) / FOUR_PI)
        X, tri = mg.icosphere(level)
        A = 0.5 * np.linalg.norm(np.cross(X[tri[:, 1]] - X[tri[:, 0]], X[tri[:, 2]] - X[tri[:, 0]]), axis=1).sum()
        flat.append(abs(A - FOUR_PI) / FOUR_PI)
    assert errs[1] < 1e-4 and errs[0] / errs[1] > 12.0, errs
    assert 3.0 < flat[0] / flat[1] < 5.0, flat
    assert errs[1] < flat[1] / 100.0


@pytest.mark.slow
def test_sphere_conductor_fourth_order(C, oracle_mod):
    """Conductor sphere R = 1 at V0 = 1 (Eq. Final1): sigma = 1 at every vertex and
    total charge 4 pi, approached at O(h^4); at level 2 the error is far below that
    of flat P0 triangles with centroid collocation on the same vertices."""
    errs = []
    for level in (1, 2):
        nodes, tri6, nv = mg.quadratic_sphere(level)
        P = C.CurvedProblem(nodes, tri6, nv)
        u = P.solve_conductor(1.0)
        errs.append([np.abs(u - 1.0).max(), abs(P.integrate(u) - FOUR_PI) / FOUR_PI])
    errs = np.array(errs)
    assert np.all(errs[1] < [1e-4, 5e-5]), errs
    assert np.all(errs[0] / errs[1] > 10.0), errs
    uf = oracle_mod.Problem(mg.sphere_mesh(2), eta=4.0, g=3).solve()
    assert errs[1, 0] < np.abs(uf - 1.0).max() / 100.0


def test_quadrature_parameters_do_not_change_the_solution(C):
    """eta = 4 with an 8x8 regular rule and eta = 2 with 12x12 (and other near-rule
    orders) give the same density to 1e-11."""
    nodes, tri6, nv = mg.quadratic_sphere(1)
    u1 = C.CurvedProblem(nodes, tri6, nv, eta=4.0, g=8, n=24, n_near=(16, 64)).solve_conductor()
    u2 = C.CurvedProblem(nodes, tri6, nv, eta=2.0, g=12, n=32, n_near=(20, 80)).solve_conductor()
    assert np.abs(u1 - u2).max() < 1e-11


def test_flat_field_reduction_to_closed_form(C, oracle_mod):
    """sum_k of the basis functions' fields G_k = the closed-form field of a
    constant density (Graglia / solid angle), off the surface: regular and
    near-singular points, down to 1e-6 R from the triangle."""
    worst = 0.0
    for a, b, c in _shaped_triangles(6, 21):
        P6 = _flat6(a, b, c)
        cc, R = C.circumcircle(a, b, c)
        n = np.cross(b - a, c - a)
        n /= np.linalg.norm(n)
        ctr = (a + b + c) / 3.0
        for x, kind in [(cc + 2.0001 * R * n, "regular"), (cc + 5.0 * R * np.array([0.6, 0.0, 0.8]), "regular"),
                        (ctr + 0.1 * R * n, "near"), (ctr - 1e-6 * R * n, "near"),
                        (0.5 * (a + b) + 0.01 * R * n, "near"), (a + 0.2 * (a - ctr), "near"),
                        (b - 1e-4 * R * n, "near")]:
            _, G = oracle_mod.tri_exact(x, a, b, c)
            _, Gk = C.pair_integrals(x, P6, kind, want_G=True)
            worst = max(worst, np.abs(Gk.sum(axis=0) - G).max() / np.abs(G).max())
    assert worst < 1e-10, worst


@pytest.mark.slow
def test_sphere_field_fourth_order(C):
    """The conductor sphere's field at 50 points inside (phi = 1, E = 0) and 50
    outside (phi = 1/r, E = x/r^3) converges at O(h^4) or better."""
    pts = mg.sphere_eval_points(1, 50, 50)
    r = np.linalg.norm(pts, axis=1)
    inside = r < 1.0
    phi_t = np.where(inside, 1.0, 1.0 / r)
    E_t = np.where(inside[:, None], 0.0, pts / r[:, None] ** 3)
    errs = []
    for level in (1, 2):
        nodes, tri6, nv = mg.quadratic_sphere(level)
        P = C.CurvedProblem(nodes, tri6, nv)
        phi, E = P.field(P.solve_conductor(), pts)
        errs.append([np.abs(phi - phi_t).max(), np.abs(E - E_t).max()])
    errs = np.array(errs)
    assert np.all(errs[1] < [5e-5, 1e-4]), errs
    assert np.all(errs[0] / errs[1] > 10.0), errs


@pytest.mark.slow
def test_conductor_inside_dielectric_sphere_curved(C, oracle_mod):
    """Eqs. Final1 + Final3 on concentric spheres: a conductor (a = 1, V0 = 1)
    inside a dielectric ball (b = 2, eps_r = 4 inside, 1 outside).  Gauss gives the
    charges Q/eps on the conductor and Q (1 - 1/eps) on the interface, with
    Q = 4 pi V0 / (1/(eps a) + (1 - 1/eps)/b).  With K' as the mean of the one-sided
    normal fields, curved P1 converges at about third order (flat P0, whose K'
    misses the curvature of its own panel, at first order) and at level 2 is far
    more accurate than flat P0 on the same vertices."""
    a, b, eps, V0 = 1.0, 2.0, 4.0, 1.0
    Q = FOUR_PI * V0 / (1.0 / (eps * a) + (1.0 - 1.0 / eps) / b)
    want = np.array([Q / eps, Q * (1.0 - 1.0 / eps)])
    regions = [{"kind": "conductor", "V0": V0}, {"kind": "dielectric", "eps_plus": 1.0, "eps_minus": eps}]
    errs = []
    for level in (1, 2):
        nodes, tri6, nv, body = mg.quadratic_bodies([mg.quadratic_sphere(level, a), mg.quadratic_sphere(level, b)])
        P = C.CurvedProblem(nodes, tri6, nv)
        u, vreg = P.solve(regions, body)
        xi, eta, w = C.duffy(C.CORNERS[0], C.CORNERS[1], C.CORNERS[2], 12)
        lam = C.linear(xi, eta)
        q = np.zeros(2)
        for T in range(P.N):
            _, J = C.surface(nodes[tri6[T]], xi, eta)
            q[body[T]] += np.sum(w * J * (lam @ u[tri6[T, :3]]))
        errs.append(np.abs(q - want) / want)
    errs = np.array(errs)
    assert np.all(errs[1] < 6e-3), errs
    assert np.all(errs[0] / errs[1] > 5.0), errs
    # flat P0 on the same two icospheres (centroid collocation)
    X1, T1 = mg.icosphere(2, a)
    X2, T2 = mg.icosphere(2, b)
    flat = mg.Mesh(np.concatenate([X1, X2]), np.concatenate([T1, T2 + len(X1)]).astype(np.int32),
                   np.concatenate([np.zeros(len(T1), np.int32), np.ones(len(T2), np.int32)]), regions)
    Pf = oracle_mod.Problem(flat, eta=4.0, g=3)
    uf = Pf.solve()
    qf = np.array([np.sum((uf[: Pf.N] * Pf.area)[flat.region == k]) for k in (0, 1)])
    assert np.all(errs[1] < np.abs(qf - want) / want / 5.0), (errs[1], np.abs(qf - want) / want)


@pytest.mark.slow
def test_floating_sphere_next_to_conductor_curved(C):
    """Eqs. Final1, Final2, Final4 on curved P1: a conductor sphere (a = 1 at V0 = 1)
    and a neutral floating sphere (a = 0.5, centres 2.5 apart).  The floating
    potential and the conductor's charge approach the method-of-images series at
    about fourth order; the floating sphere's net charge is zero to rounding."""
    from test_oracle_solve import two_sphere_images
    a1, a2, d, V1 = 1.0, 0.5, 2.5, 1.0
    V2, Q1 = two_sphere_images(a1, a2, d, V1)
    regions = [{"kind": "conductor", "V0": V1}, {"kind": "floating", "floating_id": 0, "eps_plus": 1.0}]
    errs = []
    for level in (1, 2):
        n2, t2, nv2 = mg.quadratic_sphere(level, a2)
        nodes, tri6, nv, body = mg.quadratic_bodies([mg.quadratic_sphere(level, a1),
                                                     (n2 + np.array([d, 0.0, 0.0]), t2, nv2)])
        P = C.CurvedProblem(nodes, tri6, nv)
        x, vreg = P.solve(regions, body)
        xi, eta, w = C.duffy(C.CORNERS[0], C.CORNERS[1], C.CORNERS[2], 12)
        lam = C.linear(xi, eta)
        q = np.zeros(2)
        for T in range(P.N):
            _, J = C.surface(nodes[tri6[T]], xi, eta)
            q[body[T]] += np.sum(w * J * (lam @ x[tri6[T, :3]]))
        assert abs(q[1]) < 1e-12 * abs(q[0])
        errs.append([abs(x[nv] - V2) / V2, abs(q[0] - Q1) / Q1])
    errs = np.array(errs)
    assert np.all(errs[1] < 1e-4), errs
    assert np.all(errs[0] / errs[1] > 8.0), errs

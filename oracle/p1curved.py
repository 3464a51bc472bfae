"""Plain FP64 CPU oracle for the paper's own discretisation: a mapped linear (P1)
nodal basis on curved, piecewise quadratic triangles, collocated at the vertices.

TEST INFRASTRUCTURE ONLY: only tests/ may import this module.  It shares no code
with the CUDA library; its inputs are the seeded geometry of
``paper_2003_12663_gb300.meshgen`` (``quadratic_sphere``, ``quadratic_from_flat``).

What it computes (paper sections / equations):

* the surface: triangles tau_T with a quadratic parametrisation y_T(xi, eta) over
  the reference triangle (0,0), (1,0), (0,1) through six nodes (the corners, then
  the midpoints of the edges 01, 12, 20) -- Sec. 3, first challenge;
* the density sigma_h = sum_j u_j psi_j, psi_j the mapped linear function that is
  1 at vertex j and 0 at the other vertices (Sec. 3; "piecewise (mapped) linear
  basis functions", Sec. 4);
* the matrix entries v_ij = int psi_j(y) / (4 pi |x_i - y|) dS_y of Eq. (Matrix),
  collocation points x_i = the vertices (Sec. 3), summed over the triangles that
  carry psi_j;
* the pair types of Sec. 4 for (collocation point, triangle): singular when the
  point is a node of the triangle; regular when D > eta R (D the distance from
  the point to the circumcentre of the triangle's corners, R their circumradius);
  near-singular otherwise;
* the integration of all three by the Duffy transformation (Sec. 4): regular pairs
  with a Gauss rule collapsed at a corner; singular pairs collapsed at the
  collocation point's corner; near-singular pairs after splitting the triangle at
  its point closest to the collocation point, each part collapsed at that point;
* conductor rows (Eq. Final1): sum_j v_ij u_j = V0, solved by LU (numpy/LAPACK);
* phi and E of sigma_h at points off the surface (field formula, end of Sec. 2);
* dielectric rows (Eq. Final3) with K'sigma at a vertex taken as the mean of the
  two one-sided limits of the normal field (the jump relations of Eq. ADL);
* floating conductors (Eqs. Final2, Final4), the neutrality row by Gauss's law.

The quadrature orders are not stated in the paper; the defaults here (eta = 2 with
a 12x12 regular rule, 24x24 singular, near-singular 16 points per radial piece and
64 angular)
are checked against closed forms by the tests.
"""
from __future__ import annotations

import numpy as np

FOUR_PI = 4.0 * np.pi

# the reference triangle's corners, in the order of the geometry nodes
CORNERS = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])


def gauss01(n: int):
    """n-point Gauss-Legendre rule on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def shape(xi, eta):
    """Quadratic Lagrange shape functions of the six nodes and their derivatives
    in xi and eta; arrays of shape (..., 6)."""
    l0, l1, l2 = 1.0 - xi - eta, xi, eta
    N = np.stack([l0 * (2 * l0 - 1), l1 * (2 * l1 - 1), l2 * (2 * l2 - 1),
                  4 * l0 * l1, 4 * l1 * l2, 4 * l2 * l0], axis=-1)
    # d l0 = (-1, -1), d l1 = (1, 0), d l2 = (0, 1)
    z = np.zeros_like(xi)
    dxi = np.stack([-(4 * l0 - 1), 4 * l1 - 1, z,
                    4 * (l0 - l1), 4 * l2, -4 * l2], axis=-1)
    deta = np.stack([-(4 * l0 - 1), z, 4 * l2 - 1,
                     -4 * l1, 4 * l1, 4 * (l0 - l2)], axis=-1)
    return N, dxi, deta


def linear(xi, eta):
    """The three mapped linear basis functions (1 at one corner), shape (..., 3)."""
    return np.stack([1.0 - xi - eta, xi, eta], axis=-1)


def surface(P6, xi, eta):
    """Points y (M, 3) and area elements |dy/dxi x dy/deta| (M,) of the curved
    triangle with nodes P6 (6, 3) at reference points (xi, eta)."""
    N, dxi, deta = shape(xi, eta)
    y = N @ P6
    t1 = dxi @ P6
    t2 = deta @ P6
    return y, np.linalg.norm(np.cross(t1, t2), axis=-1)


def duffy(P0, P1, P2, n: int):
    """Gauss rule on the reference sub-triangle (P0, P1, P2), collapsed at P0 (Duffy):
    (xi, eta) = P0 + s (P1 - P0) + s t (P2 - P1), weight w_s w_t s |det|.
    Returns xi, eta, w (n*n each)."""
    s, ws = gauss01(n)
    t, wt = gauss01(n)
    S, T = np.meshgrid(s, t, indexing="ij")
    W = np.outer(ws, wt) * S
    P0, P1, P2 = (np.asarray(p, dtype=np.float64) for p in (P0, P1, P2))
    e1, e2 = P1 - P0, P2 - P1
    det = abs(e1[0] * e2[1] - e1[1] * e2[0])
    pts = P0 + S[..., None] * e1 + (S * T)[..., None] * e2
    return pts[..., 0].ravel(), pts[..., 1].ravel(), (W * det).ravel()


def duffy_graded(P0, P1, P2, n: int, s_min: float, nt: int, q: float = 0.2):
    """The Duffy rule of duffy(), with the radial variable s split geometrically
    at 1, q, q^2, ... down to below s_min, n Gauss points in each piece, and nt
    points in the angular variable t: the adaptive refinement toward the collapse
    point that a near-singular pair needs (the integrand varies on the scale
    s ~ distance / size there; a skinny part needs many angular points)."""
    m = 0 if s_min >= 1.0 else min(60, int(np.ceil(np.log(s_min) / np.log(q))))
    edges = np.concatenate([[0.0], q ** np.arange(m, -1, -1.0)])
    x, w = gauss01(n)
    s = np.concatenate([lo + (hi - lo) * x for lo, hi in zip(edges[:-1], edges[1:])])
    ws = np.concatenate([(hi - lo) * w for lo, hi in zip(edges[:-1], edges[1:])])
    t, wt = gauss01(nt)
    S, T = np.meshgrid(s, t, indexing="ij")
    W = np.outer(ws, wt) * S
    P0, P1, P2 = (np.asarray(p, dtype=np.float64) for p in (P0, P1, P2))
    e1, e2 = P1 - P0, P2 - P1
    det = abs(e1[0] * e2[1] - e1[1] * e2[0])
    pts = P0 + S[..., None] * e1 + (S * T)[..., None] * e2
    return pts[..., 0].ravel(), pts[..., 1].ravel(), (W * det).ravel()


def circumcircle(a, b, c):
    """Circumcentre and circumradius of the flat triangle (a, b, c)."""
    ab, ac = b - a, c - a
    n = np.cross(ab, ac)
    cc = a + (np.dot(ac, ac) * np.cross(n, ab) + np.dot(ab, ab) * np.cross(ac, n)) / (2.0 * np.dot(n, n))
    return cc, np.linalg.norm(cc - a)


def _project_reference(p):
    """The point of the reference triangle closest to p (2,), in reference coordinates."""
    xi, eta = p
    if xi + eta > 1.0:
        d = 0.5 * (xi + eta - 1.0)
        xi, eta = xi - d, eta - d
    xi, eta = max(xi, 0.0), max(eta, 0.0)
    if xi + eta > 1.0:  # clipping may leave it outside again: onto the hypotenuse
        xi, eta = xi / (xi + eta), eta / (xi + eta)
    return np.array([xi, eta])


def closest_point(x, P6, iters: int = 30):
    """Reference coordinates of the point of the curved triangle nearest to x:
    start from the best of a sample of points, then projected Gauss-Newton steps on
    |y(xi, eta) - x|^2."""
    k = 12
    g = np.array([(i / k, j / k) for i in range(k + 1) for j in range(k + 1 - i)])
    y, _ = surface(P6, g[:, 0], g[:, 1])
    p = g[np.argmin(np.linalg.norm(y - x, axis=1))].copy()
    for _ in range(iters):
        N, dxi, deta = shape(np.array([p[0]]), np.array([p[1]]))
        F = (N @ P6)[0] - x
        J = np.stack([(dxi @ P6)[0], (deta @ P6)[0]], axis=1)  # 3 x 2
        step = np.linalg.lstsq(J, -F, rcond=None)[0]
        q = _project_reference(p + step)
        if np.linalg.norm(q - p) < 1e-15:
            break
        p = q
    return p


def pair_integrals(x, P6, kind: str, corner: int = -1, g: int = 8, n: int = 24,
                   n_near=(16, 64), want_G: bool = False):
    """(3,) vector: int lambda_k(y) / (4 pi |x - y|) dS_y over the curved triangle
    P6, for its three mapped linear functions lambda_k.
      kind "regular":  Duffy rule of order g collapsed at corner 0;
      kind "singular": x is the triangle's corner `corner`, collapsed there;
      kind "near":     split at the point closest to x, each part collapsed there,
                       its radial variable refined geometrically toward that point
                       down to a tenth of the distance over the triangle's size
                       (n_near = points per radial piece, angular points).
    With want_G (x off the triangle: regular or near kinds), also the (3, 3)
    array G[k] = int lambda_k(y) (x - y) / (4 pi |x - y|^3) dS_y, the field of
    each basis function (the field formula at the end of Sec. 2)."""
    if kind == "regular":
        parts = [(CORNERS[0], CORNERS[1], CORNERS[2], g)]
    elif kind == "singular":
        a, b, c = corner, (corner + 1) % 3, (corner + 2) % 3
        parts = [(CORNERS[a], CORNERS[b], CORNERS[c], n)]
    else:
        p = closest_point(x, P6)
        parts = [(p, CORNERS[k], CORNERS[(k + 1) % 3], n) for k in range(3)]
        yp, _ = surface(P6, p[:1], p[1:])
        size = np.max(np.linalg.norm(P6[:3] - yp[0], axis=1))
        s_min = 0.1 * np.linalg.norm(x - yp[0]) / size
    out = np.zeros(3)
    G = np.zeros((3, 3))
    for P0, P1, P2, order in parts:
        if kind == "near":
            xi, eta, w = duffy_graded(P0, P1, P2, n_near[0], s_min, n_near[1])
        else:
            xi, eta, w = duffy(P0, P1, P2, order)
        keep = w > 0.0
        if not np.any(keep):
            continue
        xi, eta, w = xi[keep], eta[keep], w[keep]
        y, J = surface(P6, xi, eta)
        d = x - y
        r = np.linalg.norm(d, axis=1)
        lam = linear(xi, eta)
        out += (w * J / r) @ lam
        if want_G:
            G += lam.T @ ((w * J / r ** 3)[:, None] * d)
    if want_G:
        return out / FOUR_PI, G / FOUR_PI
    return out / FOUR_PI


class CurvedProblem:
    """Conductor collocation system (Eq. Final1) of the P1 / curved-quadratic
    discretisation, collocation at the vertices.  The near-singular rule is exact
    to rounding on well-shaped triangles; a very skinny triangle would need more
    angular points (n_near[1]).

    nodes: (nn, 3) geometry nodes, the first nv being the triangle corners;
    tri6: (N, 6) node indices (corners, then edge midpoints 01, 12, 20)."""

    def __init__(self, nodes, tri6, nv: int, eta: float = 2.0, g: int = 12, n: int = 24,
                 n_near=(16, 64)):
        self.nodes = np.asarray(nodes, dtype=np.float64)
        self.tri6 = np.asarray(tri6, dtype=np.int64)
        self.nv = int(nv)
        self.N = len(self.tri6)
        self.eta, self.g, self.n, self.n_near = float(eta), int(g), int(n), tuple(n_near)
        assert np.all(self.tri6[:, :3] < self.nv)

    def matrix(self):
        """Dense (nv, nv) matrix v_ij of Eq. (Matrix)."""
        X = self.nodes[: self.nv]
        V = np.zeros((self.nv, self.nv))
        for T in range(self.N):
            P6 = self.nodes[self.tri6[T]]
            vt = self.tri6[T, :3]
            cc, R = circumcircle(P6[0], P6[1], P6[2])
            D = np.linalg.norm(X - cc, axis=1)
            sing = np.zeros(self.nv, dtype=bool)
            sing[vt] = True
            reg = (D > self.eta * R) & ~sing
            # regular pairs, all such collocation points at once
            xi, eta, w = duffy(CORNERS[0], CORNERS[1], CORNERS[2], self.g)
            y, J = surface(P6, xi, eta)
            idx = np.where(reg)[0]
            if len(idx):
                r = np.linalg.norm(X[idx, None, :] - y[None, :, :], axis=2)
                V[np.ix_(idx, vt)] += ((w * J)[None, :] / r) @ linear(xi, eta) / FOUR_PI
            for k in range(3):
                V[vt[k], vt] += pair_integrals(X[vt[k]], P6, "singular", corner=k, n=self.n)
            for i in np.where(~reg & ~sing)[0]:
                V[i, vt] += pair_integrals(X[i], P6, "near", n_near=self.n_near)
        return V

    def solve_conductor(self, V0: float = 1.0, V=None):
        """u at the vertices for a conductor held at V0 (Eq. Final1), by LU."""
        if V is None:
            V = self.matrix()
        return np.linalg.solve(V, np.full(self.nv, V0))

    def field(self, u, pts):
        """phi and E at points off the surface (the field formula at the end of
        Sec. 2) for vertex values u: every (point, triangle) pair by the regular
        rule if D > eta R, else by the near-singular rule."""
        pts = np.asarray(pts, dtype=np.float64).reshape(-1, 3)
        phi = np.zeros(len(pts))
        E = np.zeros((len(pts), 3))
        xi, eta, w = duffy(CORNERS[0], CORNERS[1], CORNERS[2], self.g)
        lam = linear(xi, eta)
        for T in range(self.N):
            P6 = self.nodes[self.tri6[T]]
            uT = u[self.tri6[T, :3]]
            cc, R = circumcircle(P6[0], P6[1], P6[2])
            reg = np.linalg.norm(pts - cc, axis=1) > self.eta * R
            y, J = surface(P6, xi, eta)
            dens = w * J * (lam @ uT)
            idx = np.where(reg)[0]
            if len(idx):
                d = pts[idx, None, :] - y[None, :, :]
                r = np.linalg.norm(d, axis=2)
                phi[idx] += (dens[None, :] / r).sum(axis=1) / FOUR_PI
                E[idx] += np.einsum("pq,pqc->pc", dens[None, :] / r ** 3, d) / FOUR_PI
            for i in np.where(~reg)[0]:
                S, G = pair_integrals(pts[i], P6, "near", n_near=self.n_near, want_G=True)
                phi[i] += S @ uT
                E[i] += uT @ G
        return phi, E

    def vertex_normals(self):
        """Unit normal at every vertex: the sum of the unit normals that the curved
        triangles around it have at that corner (their maps' dy/dxi x dy/deta),
        normalised.  The triangles' corners are counter-clockwise about the normal
        of the + side."""
        nrm = np.zeros((self.nv, 3))
        for T in range(self.N):
            P6 = self.nodes[self.tri6[T]]
            _, dxi, deta = shape(CORNERS[:, 0], CORNERS[:, 1])
            n = np.cross(dxi @ P6, deta @ P6)
            nrm[self.tri6[T, :3]] += n / np.linalg.norm(n, axis=1, keepdims=True)
        return nrm / np.linalg.norm(nrm, axis=1, keepdims=True)

    def _regular_rule(self):
        """Every triangle's regular-rule points Y (N, Q, 3) and weights w J (N, Q),
        the basis values (Q, 3), circumcentres (N, 3) and radii (N,)."""
        if not hasattr(self, "_rr"):
            xi, eta, w = duffy(CORNERS[0], CORNERS[1], CORNERS[2], self.g)
            Y, WJ, CC, R = [], [], [], []
            for T in range(self.N):
                P6 = self.nodes[self.tri6[T]]
                y, J = surface(P6, xi, eta)
                Y.append(y)
                WJ.append(w * J)
                c, r = circumcircle(P6[0], P6[1], P6[2])
                CC.append(c)
                R.append(r)
            self._rr = (np.array(Y), np.array(WJ), linear(xi, eta), np.array(CC), np.array(R))
        return self._rr

    def basis_fields(self, x):
        """(nv, 3): the field at x (off the surface) of every basis function psi_v:
        the regular pairs of all triangles at once, the near-singular ones one by one."""
        Y, WJ, lam, CC, R = self._regular_rule()
        out = np.zeros((self.nv, 3))
        reg = np.linalg.norm(x - CC, axis=1) > self.eta * R
        d = x - Y[reg]
        r = np.linalg.norm(d, axis=2)
        G = np.einsum("tq,qk,tqc->tkc", WJ[reg] / r ** 3, lam, d) / FOUR_PI
        np.add.at(out, self.tri6[reg, :3], G)
        for T in np.where(~reg)[0]:
            _, G = pair_integrals(x, self.nodes[self.tri6[T]], "near", n_near=self.n_near, want_G=True)
            out[self.tri6[T, :3]] += G
        return out

    def kprime_rows(self, rows, delta_rel: float = 1e-3):
        """(len(rows), nv): (K' psi_v)(x_i) for the vertices i in rows, by the jump
        relations of Eq. ADL read as Plemelj's formulas: K'sigma = (E+.n + E-.n)/2,
        the mean of the two one-sided limits of the normal field.  Each limit is the
        field at x_i +- delta n_i, extrapolated to delta -> 0 from delta and 2 delta
        (Richardson); delta = delta_rel times the mean length of the edges at x_i."""
        nrm = self.vertex_normals()
        X = self.nodes[: self.nv]
        e = np.concatenate([self.tri6[:, [0, 1]], self.tri6[:, [1, 2]], self.tri6[:, [2, 0]]])
        L = np.linalg.norm(X[e[:, 0]] - X[e[:, 1]], axis=1)
        hsum = np.bincount(e[:, 0], L, self.nv) + np.bincount(e[:, 1], L, self.nv)
        hcnt = np.bincount(e[:, 0], None, self.nv) + np.bincount(e[:, 1], None, self.nv)
        h = hsum / hcnt
        out = np.zeros((len(rows), self.nv))
        for k, i in enumerate(rows):
            n = nrm[i]
            d = delta_rel * h[i]
            f = {}
            for m in (1, 2):
                Ep = self.basis_fields(X[i] + m * d * n) @ n
                Em = self.basis_fields(X[i] - m * d * n) @ n
                f[m] = 0.5 * (Ep + Em)
            out[k] = 2.0 * f[1] - f[2]
        return out

    def solve(self, regions, body, V0_scale: float = 1.0):
        """Unknowns (u at the vertices, then V_f of each floating body) and the
        vertices' regions: the system of system() solved by LU (numpy/LAPACK)."""
        A, b, vreg = self.system(regions, body, V0_scale)
        return np.linalg.solve(A, b), vreg

    def system(self, regions, body, V0_scale: float = 1.0):
        """The collocation system (A, b, vreg) for regions
        (dicts, as for flat meshes) given per triangle by body:
          conductor rows  sum_j v_ij u_j = V0                      (Eq. Final1)
          floating rows   sum_j v_ij u_j - V_f = 0                  (Eq. Final2)
          dielectric rows (eps+ + eps-)/2 u_i + (eps+ - eps-) (K'u)_i = 0  (Eq. Final3)
          neutrality      int_{body f} sigma_h dS = 0               (Eq. Final4)
        The neutrality row uses Gauss's law on a closed conductor (no field inside):
        int eps+ (sigma/2 + K'sigma) dS = eps+ int E+.n dS = eps+ int sigma dS.
        A vertex takes the region of its triangles."""
        vreg = np.full(self.nv, -1)
        for T in range(self.N):
            for v in self.tri6[T, :3]:
                assert vreg[v] in (-1, body[T]), "a vertex on two regions"
                vreg[v] = body[T]
        kinds = [regions[r]["kind"] for r in vreg]
        fids = sorted({r["floating_id"] for r in regions if r["kind"] == "floating"})
        F = len(fids)
        n = self.nv + F
        A = np.zeros((n, n))
        b = np.zeros(n)
        cond = [i for i in range(self.nv) if kinds[i] == "conductor"]
        flo = [i for i in range(self.nv) if kinds[i] == "floating"]
        diel = [i for i in range(self.nv) if kinds[i] == "dielectric"]
        assert len(cond) + len(flo) + len(diel) == self.nv, "conductor, floating and dielectric rows only"
        if cond or flo:
            V = self.matrix()
            A[cond, : self.nv] = V[cond]
            b[cond] = [regions[vreg[i]]["V0"] * V0_scale for i in cond]
            for i in flo:
                A[i, : self.nv] = V[i]
                A[i, self.nv + fids.index(regions[vreg[i]]["floating_id"])] = -1.0
        if flo:
            xi, eta, w = duffy(CORNERS[0], CORNERS[1], CORNERS[2], self.g)
            lam = linear(xi, eta)
            for T in range(self.N):
                R = regions[body[T]]
                if R["kind"] != "floating":
                    continue
                _, J = surface(self.nodes[self.tri6[T]], xi, eta)
                A[self.nv + fids.index(R["floating_id"]), self.tri6[T, :3]] += (w * J) @ lam
        if diel:
            K = self.kprime_rows(diel)
            for k, i in enumerate(diel):
                ep, em = regions[vreg[i]]["eps_plus"], regions[vreg[i]]["eps_minus"]
                A[i] = (ep - em) * K[k]
                A[i, i] += 0.5 * (ep + em)
        return A, b, vreg

    def integrate(self, u=None):
        """int sigma_h dS (the total charge) for vertex values u, or the area if
        u is None, by the order-g rule on every curved triangle."""
        xi, eta, w = duffy(CORNERS[0], CORNERS[1], CORNERS[2], self.g)
        lam = linear(xi, eta)
        total = 0.0
        for T in range(self.N):
            _, J = surface(self.nodes[self.tri6[T]], xi, eta)
            dens = np.ones_like(xi) if u is None else lam @ u[self.tri6[T, :3]]
            total += np.sum(w * J * dens)
        return total

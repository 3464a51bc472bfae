"""Plain FP64 CPU oracle for the indirect single-layer collocation BEM.

TEST INFRASTRUCTURE ONLY: only tests/, ``__graft_entry__.smoke()`` and the CPU
legs of ``bench.py`` may import this module.  It shares no code with the CUDA
library under ``paper_2003_12663_gb300/``; the only thing both sides see are the
seeded inputs from ``paper_2003_12663_gb300.meshgen``.

What it computes (paper sections / equations):

* pair integrals S_j(x), G_j(x) of a flat triangle, closed form or by the
  Duffy-transformed Gauss rule (C part, ``bem_oracle.c``);
* the classification of Sec. 4: a pair is regular iff D > eta*R, with D the
  distance of the target to the triangle's circumcentre and R the circumradius;
* the collocation system of Eqs. (Final1)-(Final4), with thin floating sheets
  by Eq. (sheets), discretised by
  piecewise-constant sigma on flat triangles with centroid collocation (Sec. 3);
* its solution by a dense LU factorisation (LAPACK through numpy);
* phi and E at arbitrary points (field formula at the end of Sec. 2);
* the surface field on the + side, E+ = E_PV + u_i n_i / 2 (Eq. ADL read as the
  jump relation E+.n = sigma/2 + K'sigma).

Two modes for the pair integrals:
  EXACT  (0): closed form for every pair -- the plain definition of the
              discrete system (what the quadrature approximates);
  METHOD (1): the paper's steps -- regular pairs by the Duffy/Gauss rule, all
              other pairs (near-singular and singular) by the closed form, which
              is the converged limit of the paper's subdivision scheme.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import scipy.special

from . import build as _build

EXACT, METHOD = 0, 1

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_lp = ctypes.POINTER(ctypes.c_int64)
_i64 = ctypes.c_int64
_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.oracle_panel_geometry.argtypes = [_i64, _dp, _ip, _dp]
        L.oracle_tri_exact.argtypes = [_dp, _dp, _dp, _dp, ctypes.c_int, _dp, _dp]
        L.oracle_tri_quad.argtypes = [_dp, _dp, _dp, _dp, ctypes.c_int, _dp, _dp, ctypes.c_int,
                                      _dp, _dp, _dp, _dp]
        L.oracle_tri_subdivide.argtypes = [_dp, _dp, _dp, _dp, ctypes.c_int, _dp, _dp, _dp, _dp]
        L.oracle_pair_block.argtypes = [_i64, _dp, _lp, _i64, _dp, _ip, _dp, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_int, _dp, _dp, ctypes.c_int,
                                        _dp, _dp, _dp, _dp]
        L.oracle_field.argtypes = [_i64, _dp, _lp, _i64, _dp, _ip, _dp, _dp, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_int, _dp, _dp, ctypes.c_int, _dp,
                                   _dp, _dp, _dp]
        L.oracle_trace.argtypes = [_i64, _dp, ctypes.c_int, ctypes.c_double, _i64, _dp, _ip, _dp,
                                   _dp, _ip, _ip, ctypes.c_double, ctypes.c_int, _dp, _dp,
                                   ctypes.c_int, _dp, _dp] + [ctypes.c_double] * 6 + \
                                  [_i64, _dp, _ip, _ip, _dp]
        L.oracle_adjoint_trace.argtypes = [_i64, _dp, ctypes.c_int, ctypes.c_double, _i64, _i64, _dp,
                                           _ip, _dp, _dp, _ip, _ip, ctypes.c_double, ctypes.c_int,
                                           _dp, _dp, ctypes.c_int, _dp, _dp] + \
                                          [ctypes.c_double] * 6 + [_i64, _dp, _dp, _ip, _dp, _dp, _dp]
        L.oracle_adjoint_trace.restype = ctypes.c_int
        L.oracle_adjoint_rows.argtypes = [_i64, _i64, _dp, _ip, _dp, _dp, _dp, _dp, ctypes.c_double,
                                          ctypes.c_int, _dp, _dp, ctypes.c_int, _dp, _dp, _dp]
        L.oracle_tri_exact_derivs.argtypes = [_dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int, _dp, _dp]
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        L.oracle_set_threads.restype = ctypes.c_int
        _lib = L
    return _lib


class TraceParams:
    """Field-line tracing parameters (Eq. Breakdowncrit): RK4 step h in arc length,
    stop radius r_max, alpha_eff(E) = c (E - E0)^2 for E > E0 else -d, stop when
    |E| < e_floor or after max_steps steps."""

    def __init__(self, h=1e-3, r_max=10.0, c=1e-2, E0=0.5, d=0.1, e_floor=1e-12, max_steps=200000):
        self.h, self.r_max, self.c, self.E0, self.d = h, r_max, c, E0, d
        self.e_floor, self.max_steps = e_floor, max_steps

    def args(self):
        return [self.h, self.r_max, self.c, self.E0, self.d, self.e_floor, int(self.max_steps)]


def _trace_call(L, seeds, analytic, q, P, u, tp):
    seeds = _c(seeds, np.float64).reshape(-1, 3)
    K = np.zeros(L)
    st = np.zeros(L, np.int32)
    ns = np.zeros(L, np.int32)
    xe = np.zeros((L, 3))
    if P is None:
        dummy_d = np.zeros(16)
        dummy_i = np.zeros(16, np.int32)
        mesh_args = [0, _d(dummy_d), dummy_i.ctypes.data_as(_ip), _d(dummy_d), _d(dummy_d),
                     dummy_i.ctypes.data_as(_ip), dummy_i.ctypes.data_as(_ip), 4.0, 1, _d(dummy_d),
                     _d(dummy_d), 1, _d(dummy_d), _d(dummy_d)]
        keep = (dummy_d, dummy_i)
    else:
        uu = _c(u[: P.N], np.float64)
        reg = _c(P.mesh.region, np.int32)
        # bodies whose surface ends a field line; a thin sheet has no inside
        elec = np.array([1 if r["kind"] in ("conductor", "floating") else 0 for r in P.mesh.regions],
                        np.int32)
        ru, rwu, rv, rwv = P.rule
        mesh_args = [P.N, _d(P.X), P.tri.ctypes.data_as(_ip), _d(P.geom), _d(uu),
                     reg.ctypes.data_as(_ip), elec.ctypes.data_as(_ip), P.eta, len(ru), _d(ru),
                     _d(rwu), len(rv), _d(rv), _d(rwv)]
        keep = (uu, reg, elec)
    lib().oracle_trace(L, _d(seeds), int(analytic), float(q), *mesh_args, *tp.args(), _d(K),
                       st.ctypes.data_as(_ip), ns.ctypes.data_as(_ip), _d(xe))
    del keep
    return K, st, ns, xe


def _adjoint_trace_call(seeds, w, analytic, q, P, u, tp):
    """Reverse pass of the lines (C): K, status, dJ/du (explicit), dJ/dX (explicit),
    dJ/dq (analytic field) for J = sum_l w_l K_l."""
    seeds = _c(seeds, np.float64).reshape(-1, 3)
    L = len(seeds)
    w = _c(np.broadcast_to(np.asarray(w, np.float64), (L,)), np.float64)
    K = np.zeros(L)
    st = np.zeros(L, np.int32)
    gq = np.zeros(1)
    if P is None:
        dd = np.zeros(16)
        di = np.zeros(16, np.int32)
        gu = np.zeros(1)
        gX = np.zeros(3)
        args = [0, 0, _d(dd), di.ctypes.data_as(_ip), _d(dd), _d(dd), di.ctypes.data_as(_ip),
                di.ctypes.data_as(_ip), 4.0, 1, _d(dd), _d(dd), 1, _d(dd), _d(dd)]
        keep = (dd, di)
    else:
        uu = _c(u[: P.N], np.float64)
        reg = _c(P.mesh.region, np.int32)
        elec = np.array([1 if r["kind"] in ("conductor", "floating") else 0 for r in P.mesh.regions],
                        np.int32)
        gu = np.zeros(P.N)
        gX = np.zeros((len(P.X), 3))
        ru, rwu, rv, rwv = P.rule
        args = [P.N, len(P.X), _d(P.X), P.tri.ctypes.data_as(_ip), _d(P.geom), _d(uu),
                reg.ctypes.data_as(_ip), elec.ctypes.data_as(_ip), P.eta, len(ru), _d(ru), _d(rwu),
                len(rv), _d(rv), _d(rwv)]
        keep = (uu, reg, elec)
    rc = lib().oracle_adjoint_trace(L, _d(seeds), int(analytic), float(q), *args, *tp.args(), _d(w),
                                    _d(K), st.ctypes.data_as(_ip), _d(gu), _d(gX), _d(gq))
    del keep
    if rc != 0:
        raise ValueError("a line ended on another electrode or in a singular field (status 2 or -1); "
                         "the gradient is not defined there")
    return K, st, gu, gX, gq[0]


def adjoint_point_charge(seeds, w=1.0, q=1.0, tp=None):
    """dJ/dq for J = sum_l w_l K_l along the lines of E = q x/|x|^3 (reverse pass).
    Returns K, status, dJ/dq."""
    tp = tp or TraceParams()
    K, st, _, _, gq = _adjoint_trace_call(seeds, w, 1, q, None, None, tp)
    return K, st, gq


def trace_point_charge(seeds, q=1.0, tp=None):
    """Field lines of E = q x / |x|^3 (the continuum field of a unit sphere at
    potential q), for pinning the integrator and its event handling."""
    tp = tp or TraceParams()
    seeds = np.asarray(seeds, np.float64).reshape(-1, 3)
    return _trace_call(len(seeds), seeds, 1, q, None, None, tp)


def set_threads(n: int) -> int:
    """OpenMP threads of the C loops (n <= 0: unchanged); returns the previous count."""
    return lib().oracle_set_threads(int(n))


def _d(a):
    return a.ctypes.data_as(_dp)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ----------------------------------------------------------------- quadrature rules
def gauss_legendre01(n: int):
    """n-point Gauss-Legendre rule on [0,1] (numpy's Legendre routine, mapped)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return (x + 1.0) / 2.0, w / 2.0


def gauss_jacobi01_u(n: int):
    """n-point Gauss rule on [0,1] for the weight u: sum_k W_k p(u_k) = int_0^1 u p(u) du
    exactly for deg p <= 2n-1 (scipy's Gauss-Jacobi routine with beta=1, mapped)."""
    x, w = scipy.special.roots_jacobi(n, 0.0, 1.0)
    return (x + 1.0) / 2.0, w / 4.0


def far_rule(g: int):
    """The regular-pair rule: Duffy collapse at the triangle's first vertex, a
    g-point Gauss rule in the collapsed coordinate u that absorbs the Jacobian
    factor u, and g-point Gauss-Legendre in v.  Returned as (u, wu, v, wv) with
    wu = W/u because the C side multiplies the Jacobian u back in."""
    u, W = gauss_jacobi01_u(g)
    v, wv = gauss_legendre01(g)
    return u, W / u, v, wv


# ----------------------------------------------------------------- single pairs
def panel_geometry(X, tri):
    """(np, 11): n[3], area, centroid[3], circumcentre[3], circumradius."""
    X = _c(X, np.float64)
    tri = _c(tri, np.int32)
    g = np.empty((len(tri), 11))
    lib().oracle_panel_geometry(len(tri), _d(X), tri.ctypes.data_as(_ip), _d(g))
    return g


def tri_exact(x, a, b, c, self_pair: bool = False):
    x, a, b, c = (_c(v, np.float64) for v in (x, a, b, c))
    S = np.zeros(1)
    G = np.zeros(3)
    lib().oracle_tri_exact(_d(x), _d(a), _d(b), _d(c), int(self_pair), _d(S), _d(G))
    return S[0], G


def tri_exact_derivs(x, a, b, c, self_pair=False, centroid=False):
    """Derivatives of the closed form (complex step): dS[12], dG[12,3] with respect to
    x (0..2), a (3..5), b (6..8), c (9..11); centroid: x is the centroid of (a, b, c)
    and moves with them."""
    x, a, b, c = (_c(v, np.float64) for v in (x, a, b, c))
    dS = np.zeros(12)
    dG = np.zeros((12, 3))
    lib().oracle_tri_exact_derivs(_d(x), _d(a), _d(b), _d(c), int(self_pair), int(centroid), _d(dS),
                                  _d(dG))
    return dS, dG


def tri_quad(x, a, b, c, rule):
    x, a, b, c = (_c(v, np.float64) for v in (x, a, b, c))
    u, wu, v, wv = (_c(r, np.float64) for r in rule)
    S = np.zeros(1)
    G = np.zeros(3)
    lib().oracle_tri_quad(_d(x), _d(a), _d(b), _d(c), len(u), _d(u), _d(wu), len(v), _d(v),
                          _d(wv), _d(S), _d(G))
    return S[0], G


def tri_subdivide(x, a, b, c, ng: int):
    """Sec. 4 near-singular scheme (closest point, split, Duffy) with order ng."""
    x, a, b, c = (_c(v, np.float64) for v in (x, a, b, c))
    gk, gw = gauss_legendre01(ng)
    S = np.zeros(1)
    G = np.zeros(3)
    lib().oracle_tri_subdivide(_d(x), _d(a), _d(b), _d(c), ng, _d(gk), _d(gw), _d(S), _d(G))
    return S[0], G


# ----------------------------------------------------------------- blocks
class Problem:
    """Mesh + method parameters, with the per-panel geometry precomputed."""

    def __init__(self, mesh, eta: float = 4.0, g: int = 4):
        self.mesh = mesh
        self.X = _c(mesh.X, np.float64)
        self.tri = _c(mesh.tri, np.int32)
        self.geom = panel_geometry(self.X, self.tri)
        self.eta = float(eta)
        self.g = int(g)
        self.rule = tuple(_c(r, np.float64) for r in far_rule(self.g))
        self.N = len(self.tri)
        self.normals = self.geom[:, 0:3]
        self.area = self.geom[:, 3]
        self.centroids = self.geom[:, 4:7].copy()
        kinds = [r["kind"] for r in mesh.regions]
        self.kind = np.array([kinds[r] for r in mesh.region])
        self.F = mesh.n_floating

    # pair integrals for targets x all panels
    def pair_block(self, pts, self_idx=None, mode=METHOD, want_G=True):
        pts = _c(pts, np.float64).reshape(-1, 3)
        M = len(pts)
        S = np.empty((M, self.N))
        G = np.empty((M, self.N, 3)) if want_G else None
        si = None if self_idx is None else _c(self_idx, np.int64)
        u, wu, v, wv = self.rule
        lib().oracle_pair_block(M, _d(pts), None if si is None else si.ctypes.data_as(_lp), self.N,
                                _d(self.X), self.tri.ctypes.data_as(_ip), _d(self.geom), mode,
                                self.eta, len(u), _d(u), _d(wu), len(v), _d(v), _d(wv), _d(S),
                                None if G is None else _d(G))
        return S, G

    def field(self, u_sigma, pts, self_idx=None, mode=METHOD):
        """phi(x), E(x) = sum_j u_j (S_j(x), G_j(x)); a target listed in self_idx
        gets the principal value of its own panel's normal field (zero)."""
        pts = _c(pts, np.float64).reshape(-1, 3)
        M = len(pts)
        phi = np.empty(M)
        E = np.empty((M, 3))
        si = None if self_idx is None else _c(self_idx, np.int64)
        uu = _c(u_sigma[: self.N], np.float64)
        u, wu, v, wv = self.rule
        lib().oracle_field(M, _d(pts), None if si is None else si.ctypes.data_as(_lp), self.N,
                           _d(self.X), self.tri.ctypes.data_as(_ip), _d(self.geom), _d(uu), mode,
                           self.eta, len(u), _d(u), _d(wu), len(v), _d(v), _d(wv), _d(phi), _d(E))
        return phi, E

    # ------------------------------------------------------------- the system
    def region_of(self, i):
        return self.mesh.regions[self.mesh.region[i]]

    def assemble(self, mode=METHOD, block: int = 1024):
        """Dense (N+F)x(N+F) matrix of Eqs. (Final1)-(Final4) with P0 sigma and
        centroid collocation.  Row i (centroid c_i, normal n_i):
          conductor : sum_j S_ij u_j                                  = V0
          floating f: sum_j S_ij u_j - V_f                            = 0
          dielectric: (eps+ + eps-)/2 u_i + (eps+ - eps-) (K'u)_i     = 0
        with (K'u)_i = n_i . sum_j G_j(c_i) u_j (principal value, own panel 0).
        Row N+f (charge neutrality of floating conductor f, Eq. Final4, centroid
        rule, divided by the conductor's area):
          sum_{i in f} A_i eps+ (u_i/2 + (K'u)_i) / area_f             = 0
        A thin floating sheet (one surface, kind "sheet") has the potential rows
        of a floating conductor; its neutrality row takes the fields of both
        sides (Eq. sheets):
          sum_{i in f} A_i ((eps+ + eps-)/2 u_i + (eps+ - eps-) (K'u)_i) / area_f = 0
        """
        N, F = self.N, self.F
        A = np.zeros((N + F, N + F))
        regions = self.mesh.regions
        reg = self.mesh.region
        neut = np.zeros((F, N))
        area_f = np.zeros(F)
        for r0 in range(0, N, block):
            r1 = min(N, r0 + block)
            idx = np.arange(r0, r1)
            S, G = self.pair_block(self.centroids[r0:r1], idx, mode)
            Kp = np.einsum("ijk,ik->ij", G, self.normals[r0:r1])
            for ii, i in enumerate(idx):
                R = regions[reg[i]]
                if R["kind"] == "conductor":
                    A[i, :N] = S[ii]
                elif R["kind"] == "floating":
                    f = R["floating_id"]
                    A[i, :N] = S[ii]
                    A[i, N + f] = -1.0
                    row = Kp[ii].copy()
                    row[i] += 0.5
                    neut[f] += self.area[i] * R.get("eps_plus", 1.0) * row
                    area_f[f] += self.area[i]
                elif R["kind"] == "sheet":
                    f = R["floating_id"]
                    A[i, :N] = S[ii]
                    A[i, N + f] = -1.0
                    ep, em = R["eps_plus"], R["eps_minus"]
                    row = (ep - em) * Kp[ii]
                    row[i] += 0.5 * (ep + em)
                    neut[f] += self.area[i] * row
                    area_f[f] += self.area[i]
                elif R["kind"] == "dielectric":
                    ep, em = R["eps_plus"], R["eps_minus"]
                    A[i, :N] = (ep - em) * Kp[ii]
                    A[i, i] += 0.5 * (ep + em)
                else:
                    raise ValueError(R["kind"])
        for f in range(F):
            A[N + f, :N] = neut[f] / area_f[f]
        return A

    def matvec(self, x, mode=METHOD):
        """y = A x without forming A: phi and E of the density x[:N] at every centroid
        by direct summation (own panel: principal value of the normal field), then
        the row equations of assemble() -- Eqs. (Final1)-(Final4) and (sheets) --
        applied to those sums.  Costs N^2 pair integrals and O(N) memory."""
        N, F = self.N, self.F
        x = np.asarray(x, np.float64)
        phi, E = self.field(x, self.centroids, np.arange(N), mode)
        Kp = np.einsum("ij,ij->i", E, self.normals)      # (K'x)_i
        regions = self.mesh.regions
        reg = self.mesh.region
        y = np.zeros(N + F)
        neut = np.zeros(F)
        area_f = np.zeros(F)
        for i in range(N):
            R = regions[reg[i]]
            k = R["kind"]
            if k == "conductor":
                y[i] = phi[i]
            elif k == "floating":
                f = R["floating_id"]
                y[i] = phi[i] - x[N + f]
                neut[f] += self.area[i] * R.get("eps_plus", 1.0) * (0.5 * x[i] + Kp[i])
                area_f[f] += self.area[i]
            elif k == "sheet":
                f = R["floating_id"]
                ep, em = R["eps_plus"], R["eps_minus"]
                y[i] = phi[i] - x[N + f]
                neut[f] += self.area[i] * (0.5 * (ep + em) * x[i] + (ep - em) * Kp[i])
                area_f[f] += self.area[i]
            elif k == "dielectric":
                ep, em = R["eps_plus"], R["eps_minus"]
                y[i] = 0.5 * (ep + em) * x[i] + (ep - em) * Kp[i]
            else:
                raise ValueError(k)
        for f in range(F):
            y[N + f] = neut[f] / area_f[f]
        return y

    def rhs(self, V0_scale: float = 1.0):
        """Right-hand side: V0 on conductor rows, 0 elsewhere (times V0_scale)."""
        b = np.zeros(self.N + self.F)
        for i in range(self.N):
            R = self.region_of(i)
            if R["kind"] == "conductor":
                b[i] = R["V0"] * V0_scale
        return b

    def gmres(self, b, tol=1e-10, m=100, max_iters=2000, matvec=None):
        """Restarted GMRES(m) for A u = b (Saad & Schultz 1986), the cross-check of the
        LU solution: x0 = 0, right Jacobi scaling by the diagonal of A (1 where it is 0,
        the neutrality rows), Arnoldi by modified Gram-Schmidt, Givens rotations, stop
        when ||b - A u|| <= tol ||b|| (unpreconditioned 2-norm, recomputed at every
        restart).  matvec: the product (default: the matrix-free self.matvec).
        Returns u, the iteration count and the final relative residual."""
        Av = matvec or self.matvec
        n = len(b)
        A_diag = np.zeros(n)
        # the diagonal from the matrix-free product with unit vectors would cost n products;
        # read it from the row equations instead: S_ii (conductor, floating), (eps+ + eps-)/2
        # (dielectric) or 0 (neutrality rows)
        for i in range(self.N):
            R = self.region_of(i)
            if R["kind"] == "dielectric":
                A_diag[i] = 0.5 * (R["eps_plus"] + R["eps_minus"])
            else:
                a, bb, c = (self.X[self.tri[i, k]] for k in range(3))
                A_diag[i] = tri_exact(self.centroids[i], a, bb, c, self_pair=True)[0]
        dinv = np.where(A_diag != 0.0, 1.0 / np.where(A_diag != 0.0, A_diag, 1.0), 1.0)
        u = np.zeros(n)
        bn = np.linalg.norm(b)
        its = 0
        r = b - Av(u)
        rel = np.linalg.norm(r) / bn
        while rel > tol and its < max_iters:
            V = np.zeros((m + 1, n))
            H = np.zeros((m + 1, m))
            cs, sn = np.zeros(m), np.zeros(m)
            g = np.zeros(m + 1)
            beta = np.linalg.norm(r)
            V[0] = r / beta
            g[0] = beta
            k = 0
            for k in range(m):
                w = Av(dinv * V[k])
                for i in range(k + 1):
                    H[i, k] = np.dot(w, V[i])
                    w = w - H[i, k] * V[i]
                H[k + 1, k] = np.linalg.norm(w)
                if H[k + 1, k] != 0.0:
                    V[k + 1] = w / H[k + 1, k]
                for i in range(k):       # earlier rotations on the new column
                    t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                    H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                    H[i, k] = t
                den = np.hypot(H[k, k], H[k + 1, k])
                cs[k], sn[k] = H[k, k] / den, H[k + 1, k] / den
                H[k, k], H[k + 1, k] = den, 0.0
                g[k + 1] = -sn[k] * g[k]
                g[k] = cs[k] * g[k]
                its += 1
                if abs(g[k + 1]) <= tol * bn or its >= max_iters:
                    break
            kk = k + 1
            y = np.linalg.solve(np.triu(H[:kk, :kk]), g[:kk])
            u = u + dinv * (V[:kk].T @ y)
            r = b - Av(u)
            rel = np.linalg.norm(r) / bn
        return u, its, rel

    def solve(self, mode=METHOD, V0_scale: float = 1.0, A=None):
        """u = A^{-1} b by LU with partial pivoting (LAPACK getrf/getrs via numpy)."""
        if A is None:
            A = self.assemble(mode)
        return np.linalg.solve(A, self.rhs(V0_scale))

    def surface_field(self, u_sigma, mode=METHOD):
        """E on the + side at every centroid: E_PV(c_i) + u_i n_i / 2."""
        _, E = self.field(u_sigma, self.centroids, np.arange(self.N), mode)
        return E + 0.5 * u_sigma[: self.N, None] * self.normals

    def adjoint(self, u_sigma, seeds, w, tp=None, A=None):
        """Gradient of J = sum_l w_l K_l (K_l the breakdown integral of line l, Eq.
        Breakdowncrit, in the field of u_sigma, which must solve this system for the
        mesh's V0) with respect to the vertex coordinates, the conductor potentials and
        the permittivities.  A hand-written reverse pass, in order:
          1. reverse of every traced RK4 sub-step, with the implicit-function terms of
             located events (C, oracle_adjoint_trace): dJ/du and the explicit dJ/dX
             through the panel geometry of the field along the lines;
          2. the adjoint system A^T mu = dJ/du (dense LU of the assembled matrix);
          3. dJ/dtheta += mu^T (db/dtheta - dA/dtheta u): the pair integrals of every
             row differentiated with respect to both triangles' vertices (C,
             oracle_adjoint_rows), the variation of the row normals n_i, and the
             neutrality weights A_i / area_f;
          4. dJ/dV0 (conductor rows of b) and dJ/deps (row equations).
        Returns K, gX [nv,3], gV0 [nregions], geps [nregions, 2] (eps+, eps-)."""
        tp = tp or TraceParams()
        N, F = self.N, self.F
        u = np.asarray(u_sigma, np.float64)
        K, st, gu, gX_line, _ = _adjoint_trace_call(seeds, w, 0, 0.0, self, u, tp)
        if A is None:
            A = self.assemble()
        mu = np.linalg.solve(A.T, np.concatenate([gu, np.zeros(F)]))
        regions, reg = self.mesh.regions, self.mesh.region
        # K'u at every centroid (principal value), and the field without the own panel
        _, E = self.field(u, self.centroids, np.arange(N))
        Kp = np.einsum("ij,ij->i", E, self.normals)
        E_other = E.copy()
        for i in range(N):
            a, b, c = (self.X[self.tri[i, k]] for k in range(3))
            _, Gii = tri_exact(self.centroids[i], a, b, c, self_pair=True)
            E_other[i] -= u[i] * Gii
        area_f = np.zeros(F)
        for i in range(N):
            R = regions[reg[i]]
            if R["kind"] in ("floating", "sheet"):
                area_f[R["floating_id"]] += self.area[i]
        # row weights: alpha on S_j(c_i), beta on n_i . G_j(c_i)
        alpha = np.zeros(N)
        beta = np.zeros(N)
        T = np.zeros(N)          # neutrality summand per unit area (Eqs. Final4, sheets)
        for i in range(N):
            R = regions[reg[i]]
            k = R["kind"]
            if k == "conductor":
                alpha[i] = mu[i]
            elif k in ("floating", "sheet"):
                f = R["floating_id"]
                ep = R.get("eps_plus", 1.0)
                em = R.get("eps_minus", 0.0) if k == "sheet" else 0.0
                alpha[i] = mu[i]
                beta[i] = mu[N + f] * self.area[i] * (ep - em) / area_f[f]
                T[i] = 0.5 * (ep + em) * u[i] + (ep - em) * Kp[i]
            elif k == "dielectric":
                beta[i] = mu[i] * (R["eps_plus"] - R["eps_minus"])
        gX_rows = np.zeros((len(self.X), 3))
        ru, rwu, rv, rwv = self.rule
        uu = _c(u[:N], np.float64)
        lib().oracle_adjoint_rows(N, len(self.X), _d(self.X), self.tri.ctypes.data_as(_ip), _d(self.geom),
                                  _d(uu), _d(_c(alpha, np.float64)), _d(_c(beta, np.float64)), self.eta,
                                  len(ru), _d(ru), _d(rwu), len(rv), _d(rv), _d(rwv), _d(gX_rows))
        # value R_f of every neutrality row (Eq. Final4 / sheets) at u
        Rf = np.zeros(F)
        for i in range(N):
            R = regions[reg[i]]
            if R["kind"] in ("floating", "sheet"):
                f = R["floating_id"]
                Rf[f] += self.area[i] * T[i] / area_f[f]
        gX_geo = np.zeros((len(self.X), 3))
        for i in range(N):
            a, b, c = (self.X[self.tri[i, k]] for k in range(3))
            n = self.normals[i]
            # variation of n_i = w / |w|, w = (b - a) x (c - a), in beta_i n_i . E_i (own
            # panel excluded: n_i . G_ii is 0 for every shape): with
            # p = beta (I - n n^T) E / |w|, d(p.w) = (p x (c-b)).da + ((c-a) x p).db + (p x (b-a)).dc
            if beta[i] != 0.0:
                e = E_other[i]
                pvec = beta[i] * (e - n * np.dot(n, e)) / (2.0 * self.area[i])
                gX_geo[self.tri[i, 0]] += np.cross(pvec, c - b)
                gX_geo[self.tri[i, 1]] += np.cross(c - a, pvec)
                gX_geo[self.tri[i, 2]] += np.cross(pvec, b - a)
            # the weights A_i / area_f of a neutrality row: d(sum_i A_i T_i / area_f)
            # = sum_i (T_i - R_f) dA_i / area_f, with dA/dv_k = n x (v_{k+2} - v_{k+1}) / 2
            R = regions[reg[i]]
            if R["kind"] in ("floating", "sheet"):
                f = R["floating_id"]
                coef = mu[N + f] * (T[i] - Rf[f]) / area_f[f]
                dA = 0.5 * np.array([np.cross(n, c - b), np.cross(n, a - c), np.cross(n, b - a)])
                for kk in range(3):
                    gX_geo[self.tri[i, kk]] += coef * dA[kk]
        gX = gX_line - gX_rows - gX_geo
        # conductor potentials: b_i = V0 of the row's region
        nreg = len(regions)
        gV0 = np.zeros(nreg)
        geps = np.zeros((nreg, 2))
        for i in range(N):
            r = reg[i]
            R = regions[r]
            k = R["kind"]
            if k == "conductor":
                gV0[r] += mu[i]
            elif k == "dielectric":
                geps[r, 0] -= mu[i] * (0.5 * u[i] + Kp[i])
                geps[r, 1] -= mu[i] * (0.5 * u[i] - Kp[i])
            elif k == "floating":
                f = R["floating_id"]
                geps[r, 0] -= mu[N + f] * self.area[i] * (0.5 * u[i] + Kp[i]) / area_f[f]
            elif k == "sheet":
                f = R["floating_id"]
                geps[r, 0] -= mu[N + f] * self.area[i] * (0.5 * u[i] + Kp[i]) / area_f[f]
                geps[r, 1] -= mu[N + f] * self.area[i] * (0.5 * u[i] - Kp[i]) / area_f[f]
        return K, gX, gV0, geps

    def trace(self, u_sigma, seeds, tp=None):
        """Field lines and K = int alpha_eff(|E|) ds (Eq. Breakdowncrit) in the field
        of sigma (the method's pair integrals).  Returns K, status, nsteps, xend."""
        tp = tp or TraceParams()
        seeds = np.asarray(seeds, np.float64).reshape(-1, 3)
        return _trace_call(len(seeds), seeds, 0, 0.0, self, u_sigma, tp)

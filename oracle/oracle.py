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


def trace_point_charge(seeds, q=1.0, tp=None):
    """Field lines of E = q x / |x|^3 (the continuum field of a unit sphere at
    potential q), for pinning the integrator and its event handling."""
    tp = tp or TraceParams()
    seeds = np.asarray(seeds, np.float64).reshape(-1, 3)
    return _trace_call(len(seeds), seeds, 1, q, None, None, tp)


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

    def rhs(self, V0_scale: float = 1.0):
        """Right-hand side: V0 on conductor rows, 0 elsewhere (times V0_scale)."""
        b = np.zeros(self.N + self.F)
        for i in range(self.N):
            R = self.region_of(i)
            if R["kind"] == "conductor":
                b[i] = R["V0"] * V0_scale
        return b

    def solve(self, mode=METHOD, V0_scale: float = 1.0, A=None):
        """u = A^{-1} b by LU with partial pivoting (LAPACK getrf/getrs via numpy)."""
        if A is None:
            A = self.assemble(mode)
        return np.linalg.solve(A, self.rhs(V0_scale))

    def surface_field(self, u_sigma, mode=METHOD):
        """E on the + side at every centroid: E_PV(c_i) + u_i n_i / 2."""
        _, E = self.field(u_sigma, self.centroids, np.arange(self.N), mode)
        return E + 0.5 * u_sigma[: self.N, None] * self.normals

    def trace(self, u_sigma, seeds, tp=None):
        """Field lines and K = int alpha_eff(|E|) ds (Eq. Breakdowncrit) in the field
        of sigma (the method's pair integrals).  Returns K, status, nsteps, xend."""
        tp = tp or TraceParams()
        seeds = np.asarray(seeds, np.float64).reshape(-1, 3)
        return _trace_call(len(seeds), seeds, 0, 0.0, self, u_sigma, tp)

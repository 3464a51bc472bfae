/*
 * bem_oracle.c -- plain FP64 CPU oracle for the panel-interaction evaluation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the CPU
 * legs of bench.py may load this library.  It shares no code, header, table or
 * constant generator with the CUDA library; the quadrature rule it uses is
 * generated on the Python side of the oracle and passed in as arrays.
 *
 * Notation follows the paper: a target point x, flat triangles tau_j with
 * vertices (a, b, c) ordered counter-clockwise about the unit normal n, which
 * points to the "+" side.  All integrals carry the 1/(4 pi) of Eq. (SL):
 *
 *   S_j(x) = 1/(4 pi) \int_{tau_j} 1/|x-y| dS_y                      (Eq. SL)
 *   G_j(x) = 1/(4 pi) \int_{tau_j} (x-y)/|x-y|^3 dS_y     (field formula, Sec. 2)
 *
 * so that phi = sum_j u_j S_j and E = sum_j u_j G_j for piecewise-constant
 * sigma = u_j on tau_j (Sec. 3).
 *
 * Functions:
 *   oracle_panel_geometry   normal, area, centroid, circumcentre, circumradius
 *   oracle_tri_exact        closed-form S and G (potential of a uniform density on
 *                           a polygon, its gradient, and the triangle solid angle)
 *   oracle_tri_quad         Duffy-transformed Gauss product rule (Sec. 4)
 *   oracle_tri_subdivide    the paper's near-singular scheme: split at the closest
 *                           point, Duffy on each piece, geometric refinement toward it
 *   oracle_pair_block       S and G for a block of targets x all panels, with the
 *                           classification D > eta R of Sec. 4
 *   oracle_field            phi and E by direct summation
 *   oracle_trace            RK4 field-line tracing with the breakdown integral (Eq. 1)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct { double x, y, z; } vec;

static vec mk(const double* p) { vec r = {p[0], p[1], p[2]}; return r; }
static vec add(vec a, vec b) { vec r = {a.x + b.x, a.y + b.y, a.z + b.z}; return r; }
static vec sub(vec a, vec b) { vec r = {a.x - b.x, a.y - b.y, a.z - b.z}; return r; }
static vec scl(vec a, double s) { vec r = {a.x * s, a.y * s, a.z * s}; return r; }
static double dot(vec a, vec b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static vec cross(vec a, vec b) {
    vec r = {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
    return r;
}
static double norm(vec a) { return sqrt(dot(a, a)); }

/* ------------------------------------------------------------------ geometry */
/* Per panel 11 doubles: n[3], area, centroid[3], circumcentre[3], circumradius.
 * Circumcentre and circumradius are what the classification of Sec. 4 uses. */
void oracle_panel_geometry(int64_t np, const double* X, const int32_t* tri, double* geom)
{
    for (int64_t j = 0; j < np; ++j) {
        vec a = mk(X + 3 * (int64_t)tri[3 * j + 0]);
        vec b = mk(X + 3 * (int64_t)tri[3 * j + 1]);
        vec c = mk(X + 3 * (int64_t)tri[3 * j + 2]);
        vec u = sub(b, a), v = sub(c, a);
        vec w = cross(u, v);
        double w2 = dot(w, w);
        double wn = sqrt(w2);
        vec n = scl(w, 1.0 / wn);
        vec ctr = scl(add(add(a, b), c), 1.0 / 3.0);
        /* circumcentre: a + (|u|^2 (v x w) + |v|^2 (w x u)) / (2 |w|^2) */
        vec cc = add(a, scl(add(scl(cross(v, w), dot(u, u)), scl(cross(w, u), dot(v, v))), 0.5 / w2));
        double* g = geom + 11 * j;
        g[0] = n.x; g[1] = n.y; g[2] = n.z;
        g[3] = 0.5 * wn;
        g[4] = ctr.x; g[5] = ctr.y; g[6] = ctr.z;
        g[7] = cc.x; g[8] = cc.y; g[9] = cc.z;
        g[10] = norm(sub(cc, a));
    }
}

/* ------------------------------------------------------------- closed form */
/*
 * Exact S and G of one flat triangle at x.
 *
 * With h = (x-a).n the height of x over the plane, and for every edge i from
 * p0 to p1 (unit tangent t, in-plane outward edge normal m = t x n):
 *   s0 = (p0-x).t, s1 = (p1-x).t, r0 = |p0-x|, r1 = |p1-x|,
 *   d  = (p0-x).m      (signed distance of x's projection to the edge line),
 *   f  = \int_edge dl/|x-y| = ln((r1+s1)/(r0+s0))   (= ln((r0-s0)/(r1-s1))).
 * The signed solid angle (Van Oosterom & Strackee) with A_i = v_i - x is
 *   Omega = 2 atan2(A_0.(A_1 x A_2), |A_0||A_1||A_2| + (A_0.A_1)|A_2| + (A_0.A_2)|A_1| + (A_1.A_2)|A_0|),
 * negative on the + side.  Then
 *   4 pi S = sum_i d_i f_i + h Omega,     4 pi G = sum_i m_i f_i - Omega n.
 * The in-plane part of G comes from the divergence theorem in the plane; the
 * normal part is the solid angle.  self != 0 marks x as the panel's own
 * centroid: the principal value is taken, i.e. the normal part of G is 0.
 */
void oracle_tri_exact(const double* xp, const double* ap, const double* bp, const double* cp,
                      int self, double* S, double* G)
{
    vec x = mk(xp);
    vec v[3] = {mk(ap), mk(bp), mk(cp)};
    vec w = cross(sub(v[1], v[0]), sub(v[2], v[0]));
    vec n = scl(w, 1.0 / norm(w));
    double h = dot(sub(x, v[0]), n);
    double sum_df = 0.0;
    vec gin = {0.0, 0.0, 0.0};
    for (int i = 0; i < 3; ++i) {
        vec p0 = v[i], p1 = v[(i + 1) % 3];
        vec e = sub(p1, p0);
        vec t = scl(e, 1.0 / norm(e));
        vec m = cross(t, n);
        double s0 = dot(sub(p0, x), t), s1 = dot(sub(p1, x), t);
        double r0 = norm(sub(p0, x)), r1 = norm(sub(p1, x));
        double d = dot(sub(p0, x), m);
        double f;
        if (s0 >= 0.0)
            f = log((r1 + s1) / (r0 + s0));
        else if (s1 <= 0.0)
            f = log((r0 - s0) / (r1 - s1));
        else
            f = log((r1 + s1) * (r0 - s0) / (d * d + h * h));
        if (d != 0.0) sum_df += d * f;
        gin = add(gin, scl(m, f));
    }
    double omega = 0.0;
    if (!self) {
        vec A0 = sub(v[0], x), A1 = sub(v[1], x), A2 = sub(v[2], x);
        double l0 = norm(A0), l1 = norm(A1), l2 = norm(A2);
        double num = dot(A0, cross(A1, A2));
        double den = l0 * l1 * l2 + dot(A0, A1) * l2 + dot(A0, A2) * l1 + dot(A1, A2) * l0;
        omega = 2.0 * atan2(num, den);
    }
    const double k = 1.0 / (4.0 * M_PI);
    *S = k * (sum_df + h * omega);
    vec g = sub(gin, scl(n, omega));
    G[0] = k * g.x; G[1] = k * g.y; G[2] = k * g.z;
}

/* ------------------------------------------------------------- quadrature */
/*
 * Duffy-transformed Gauss product rule on one triangle (Sec. 4: "all three types
 * of pairs can be integrated by using the Duffy transformation").  The square
 * (u,v) in [0,1]^2 is mapped onto the triangle, collapsing the edge u = 0 onto
 * vertex a:
 *     y(u,v) = a + u (b - a) + u v (c - b),    dS_y = 2A u du dv.
 * The rule (nu nodes in u, nv in v, weights over [0,1]) is supplied by the
 * caller; with the factor u kept in the integrand, the weight of node (k,l) is
 * 2A u_k wu_k wv_l.
 */
void oracle_tri_quad(const double* xp, const double* ap, const double* bp, const double* cp,
                     int nu, const double* uk, const double* wu, int nv, const double* vl,
                     const double* wv, double* S, double* G)
{
    vec x = mk(xp), a = mk(ap), b = mk(bp), c = mk(cp);
    vec ab = sub(b, a), bc = sub(c, b);
    double A2 = norm(cross(ab, sub(c, a)));
    double s = 0.0;
    vec g = {0.0, 0.0, 0.0};
    for (int k = 0; k < nu; ++k) {
        for (int l = 0; l < nv; ++l) {
            vec y = add(a, add(scl(ab, uk[k]), scl(bc, uk[k] * vl[l])));
            double w = A2 * uk[k] * wu[k] * wv[l];
            vec d = sub(x, y);
            double r = norm(d);
            s += w / r;
            g = add(g, scl(d, w / (r * r * r)));
        }
    }
    const double kk = 1.0 / (4.0 * M_PI);
    *S = kk * s;
    G[0] = kk * g.x; G[1] = kk * g.y; G[2] = kk * g.z;
}

/* closest point of triangle (a,b,c) to x, by the barycentric region test */
static vec closest_point(vec x, vec a, vec b, vec c)
{
    vec ab = sub(b, a), ac = sub(c, a), ax = sub(x, a);
    double d1 = dot(ab, ax), d2 = dot(ac, ax);
    if (d1 <= 0.0 && d2 <= 0.0) return a;
    vec bx = sub(x, b);
    double d3 = dot(ab, bx), d4 = dot(ac, bx);
    if (d3 >= 0.0 && d4 <= d3) return b;
    double vc = d1 * d4 - d3 * d2;
    if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) return add(a, scl(ab, d1 / (d1 - d3)));
    vec cx = sub(x, c);
    double d5 = dot(ab, cx), d6 = dot(ac, cx);
    if (d6 >= 0.0 && d5 <= d6) return c;
    double vb = d5 * d2 - d1 * d6;
    if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) return add(a, scl(ac, d2 / (d2 - d6)));
    double va = d3 * d6 - d5 * d4;
    if (va <= 0.0 && (d4 - d3) >= 0.0 && (d5 - d6) >= 0.0)
        return add(b, scl(sub(c, b), (d4 - d3) / ((d4 - d3) + (d5 - d6))));
    double den = 1.0 / (va + vb + vc);
    return add(a, add(scl(ab, vb * den), scl(ac, vc * den)));
}

/* Duffy rule on the sub-triangle (p, q1, q2) collapsed at p, with the radial
 * coordinate u split geometrically into [0, 2^-levels] and [2^-(k+1), 2^-k]. */
static void duffy_at(vec x, vec p, vec q1, vec q2, int levels, int ng, const double* gk,
                     const double* gw, double* s, vec* g)
{
    double A2 = norm(cross(sub(q1, p), sub(q2, p)));
    if (A2 == 0.0) return;
    vec e1 = sub(q1, p), e12 = sub(q2, q1);
    for (int lev = 0; lev <= levels; ++lev) {
        double hi = ldexp(1.0, -lev);
        double lo = (lev == levels) ? 0.0 : ldexp(1.0, -lev - 1);
        for (int k = 0; k < ng; ++k) {
            double u = lo + (hi - lo) * gk[k];
            double wu = (hi - lo) * gw[k];
            for (int l = 0; l < ng; ++l) {
                double v = gk[l];
                /* x - y formed as (x - p) - u e, so that tiny u is not lost to rounding */
                vec d = sub(sub(x, p), scl(add(e1, scl(e12, v)), u));
                double w = A2 * u * wu * gw[l];
                double r = norm(d);
                *s += w / r;
                *g = add(*g, scl(d, w / (r * r * r)));
            }
        }
    }
}

/*
 * The paper's near-singular scheme (Sec. 4): find the point p* of the triangle
 * closest to x, split the triangle into the pieces that have p* as a corner
 * (three for an interior point, two on an edge, one at a vertex) and integrate
 * each piece with a Duffy rule collapsed at p*.  The paper calls the scheme
 * adaptive without fixing its refinement; here the radial coordinate of every
 * piece is refined geometrically toward p* until the smallest cell is no larger
 * than the distance |x - p*| (gauss-legendre order ng on every cell).
 */
void oracle_tri_subdivide(const double* xp, const double* ap, const double* bp, const double* cp,
                          int ng, const double* gk, const double* gw, double* S, double* G)
{
    vec x = mk(xp), a = mk(ap), b = mk(bp), c = mk(cp);
    vec p = closest_point(x, a, b, c);
    double dist = norm(sub(x, p));
    double diam = fmax(norm(sub(b, a)), fmax(norm(sub(c, b)), norm(sub(a, c))));
    int levels = 0;
    while (levels < 60 && ldexp(diam, -levels) > dist) ++levels;
    double s = 0.0;
    vec g = {0.0, 0.0, 0.0};
    vec v[3] = {a, b, c};
    for (int i = 0; i < 3; ++i)  /* degenerate pieces (p on an edge or vertex) have zero area */
        duffy_at(x, p, v[i], v[(i + 1) % 3], levels, ng, gk, gw, &s, &g);
    const double kk = 1.0 / (4.0 * M_PI);
    *S = kk * s;
    G[0] = kk * g.x; G[1] = kk * g.y; G[2] = kk * g.z;
}

/* ------------------------------------------------------------- pair blocks */
/* mode: 0 = closed form for every pair (the plain definition of the discrete system);
 *       1 = the method: regular pairs (D > eta R, Sec. 4) by the Duffy rule,
 *           all other pairs by the closed form. */
static void pair(int mode, double eta, const double* x, int self, const double* X,
                 const int32_t* t, const double* geom, int nu, const double* uk, const double* wu,
                 int nv, const double* vl, const double* wv, double* S, double* G)
{
    const double* a = X + 3 * (int64_t)t[0];
    const double* b = X + 3 * (int64_t)t[1];
    const double* c = X + 3 * (int64_t)t[2];
    if (mode == 1 && !self) {
        double dx = x[0] - geom[7], dy = x[1] - geom[8], dz = x[2] - geom[9];
        double D = sqrt(dx * dx + dy * dy + dz * dz);
        if (D > eta * geom[10]) {
            oracle_tri_quad(x, a, b, c, nu, uk, wu, nv, vl, wv, S, G);
            return;
        }
    }
    oracle_tri_exact(x, a, b, c, self, S, G);
}

/* S[M][np] and (if G != NULL) G[M][np][3] for targets pts[M][3].  self_idx[i]
 * (nullable) is the panel whose centroid target i is, or -1. */
void oracle_pair_block(int64_t M, const double* pts, const int64_t* self_idx, int64_t np,
                       const double* X, const int32_t* tri, const double* geom, int mode,
                       double eta, int nu, const double* uk, const double* wu, int nv,
                       const double* vl, const double* wv, double* S, double* G)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < M; ++i) {
        for (int64_t j = 0; j < np; ++j) {
            double s, g[3];
            int self = self_idx ? (self_idx[i] == j) : 0;
            pair(mode, eta, pts + 3 * i, self, X, tri + 3 * j, geom + 11 * j, nu, uk, wu, nv, vl,
                 wv, &s, g);
            S[i * np + j] = s;
            if (G) {
                G[(i * np + j) * 3 + 0] = g[0];
                G[(i * np + j) * 3 + 1] = g[1];
                G[(i * np + j) * 3 + 2] = g[2];
            }
        }
    }
}

/* phi[M], E[M][3] = sum_j u_j (S_j, G_j) at pts.  Same conventions as above. */
void oracle_field(int64_t M, const double* pts, const int64_t* self_idx, int64_t np,
                  const double* X, const int32_t* tri, const double* geom, const double* u,
                  int mode, double eta, int nu, const double* uk, const double* wu, int nv,
                  const double* vl, const double* wv, double* phi, double* E)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < M; ++i) {
        double p = 0.0, e[3] = {0.0, 0.0, 0.0};
        for (int64_t j = 0; j < np; ++j) {
            double s, g[3];
            int self = self_idx ? (self_idx[i] == j) : 0;
            pair(mode, eta, pts + 3 * i, self, X, tri + 3 * j, geom + 11 * j, nu, uk, wu, nv, vl,
                 wv, &s, g);
            p += u[j] * s;
            e[0] += u[j] * g[0];
            e[1] += u[j] * g[1];
            e[2] += u[j] * g[2];
        }
        phi[i] = p;
        E[3 * i + 0] = e[0];
        E[3 * i + 1] = e[1];
        E[3 * i + 2] = e[2];
    }
}

/* ------------------------------------------------------------- field lines */
/*
 * Breakdown criterion, Eq. (Breakdowncrit): K = int_gamma alpha_eff(|E|) ds along a
 * field line gamma, traced from a seed on an electrode.
 *
 * The line follows dx/ds = s0 E/|E| (arc length s), s0 = sign(E.n) at the seed with
 * n the normal of the triangle whose centroid is nearest to the seed, and carries K
 * as an extra state, dK/ds = alpha_eff(|E(x)|), with
 *     alpha_eff(E) = c (E - E0)^2  for E > E0,   -d  otherwise.
 * Classical RK4 with step h advances (x, K).  Because alpha_eff jumps at E = E0, the
 * integrand branch ("side") is part of the state: inside a step every stage uses the
 * branch of the current side.  When the end of a step lands on the other side, the
 * crossing is located on the RK4 step itself, g(sig) = |E(x(sig))| - E0 with x(sig)
 * the end of an RK4 step of length sig, by the Illinois variant of regula falsi; the
 * step is split there and the side flips.  Terminal events are located the same way:
 * |x| = r_max (status 1), entering another electrode (status 2: the solid-angle sum
 * of that electrode's triangles, sum_j G_j.n_j with unit density, falls below -1/2;
 * -1 inside a closed body, 0 outside), |E| < e_floor (status 4, at a step start),
 * max_steps full steps (status 3), a non-finite field at a step start (status -1: the
 * flat-triangle field is singular on edges and vertices).
 */
typedef struct {
    int analytic;         /* 1: field of a point charge q at the origin, E = q x/|x|^3 */
    double q;
    int64_t np;
    const double* X;
    const int32_t* tri;
    const double* geom;
    const double* u;
    const int32_t* region;
    const int32_t* electrode; /* per region: 1 for conductor and floating bodies */
    double eta;
    int nu, nv;
    const double *uk, *wu, *vl, *wv;
} fsrc;

typedef struct {
    double h, r_max, c, E0, d, e_floor;
    int64_t max_steps;
} tparams;

static void field_pt(const fsrc* F, vec x, int seed_region, vec* E, double* ind)
{
    if (F->analytic) {
        double r = norm(x);
        *E = scl(x, F->q / (r * r * r));
        *ind = 0.0;
        return;
    }
    double xp[3] = {x.x, x.y, x.z};
    vec e = {0.0, 0.0, 0.0};
    double s_ind = 0.0;
    for (int64_t j = 0; j < F->np; ++j) {
        double s, g[3];
        pair(1, F->eta, xp, 0, F->X, F->tri + 3 * j, F->geom + 11 * j, F->nu, F->uk, F->wu, F->nv,
             F->vl, F->wv, &s, g);
        e.x += F->u[j] * g[0];
        e.y += F->u[j] * g[1];
        e.z += F->u[j] * g[2];
        int rj = F->region[j];
        if (rj != seed_region && F->electrode[rj]) {
            const double* n = F->geom + 11 * j;
            s_ind += g[0] * n[0] + g[1] * n[1] + g[2] * n[2];
        }
    }
    *E = e;
    *ind = s_ind;
}

static double alpha_eff(const tparams* P, double Em, int side)
{
    return side > 0 ? P->c * (Em - P->E0) * (Em - P->E0) : -P->d;
}

/* one RK4 step of length s from (x, K) on branch side; returns the end state */
static void rk4_step(const fsrc* F, const tparams* P, int seed_region, double s0, int side, vec x,
                     double K, double s, vec* x1, double* K1)
{
    vec k[4];
    double a[4];
    vec y = x;
    for (int st = 0; st < 4; ++st) {
        vec E;
        double ind;
        field_pt(F, y, seed_region, &E, &ind);
        double Em = norm(E);
        k[st] = scl(E, s0 / Em);
        a[st] = alpha_eff(P, Em, side);
        if (st < 3) y = add(x, scl(k[st], st < 2 ? 0.5 * s : s));
    }
    *x1 = add(x, scl(add(add(k[0], scl(add(k[1], k[2]), 2.0)), k[3]), s / 6.0));
    *K1 = K + s / 6.0 * (a[0] + 2.0 * (a[1] + a[2]) + a[3]);
}

enum { EV_ALPHA = 0, EV_RMAX = 1, EV_ELECTRODE = 2 };

/* event function of kind ev at the end of an RK4 step of length sig */
static double event_g(const fsrc* F, const tparams* P, int seed_region, double s0, int side, vec x,
                      double K, double sig, int ev)
{
    vec x1, E;
    double K1, ind;
    rk4_step(F, P, seed_region, s0, side, x, K, sig, &x1, &K1);
    if (ev == EV_RMAX) return norm(x1) - P->r_max;
    field_pt(F, x1, seed_region, &E, &ind);
    if (ev == EV_ALPHA) return norm(E) - P->E0;
    return ind + 0.5;
}

/* Illinois regula falsi on [0, b] where g(0) = ga and g(b) = gb differ in sign.
 * The event is tested at the end of the step (g(b) on the far side, or zero: a root
 * at b); if g(0) is already on that side (or zero) there is no crossing inside the
 * step -- the event condition held where the sub-step starts -- and the event is
 * located at 0. */
static double illinois(const fsrc* F, const tparams* P, int seed_region, double s0, int side, vec x,
                       double K, double b, double ga, double gb, int ev)
{
    if (gb == 0.0) return b;
    if (ga == 0.0 || (ga > 0.0) == (gb > 0.0)) return 0.0;
    double a = 0.0, c = b;
    int last = 0;
    for (int it = 0; it < 100; ++it) {
        c = (ga * b - gb * a) / (ga - gb);
        double gc = event_g(F, P, seed_region, s0, side, x, K, c, ev);
        if (gc == 0.0) break;
        if ((gc > 0.0) == (gb > 0.0)) {
            b = c; gb = gc;
            if (last == -1) ga *= 0.5;
            last = -1;
        } else {
            a = c; ga = gc;
            if (last == 1) gb *= 0.5;
            last = 1;
        }
        if (b - a <= 1e-14 * P->h) break;
    }
    return c;
}

static void trace_one(const fsrc* F, const tparams* P, const double* seed, double* K_out,
                      int32_t* status, int32_t* nsteps, double* xend)
{
    vec x = mk(seed);
    double K = 0.0;
    int seed_region = -1;
    double s0 = 1.0;
    vec E;
    double ind;
    field_pt(F, x, -2, &E, &ind);
    if (!F->analytic) {
        int64_t best = 0;
        double bd = 1e300;
        for (int64_t j = 0; j < F->np; ++j) {
            const double* c = F->geom + 11 * j + 4;
            double dd = (x.x - c[0]) * (x.x - c[0]) + (x.y - c[1]) * (x.y - c[1]) + (x.z - c[2]) * (x.z - c[2]);
            if (dd < bd) { bd = dd; best = j; }
        }
        seed_region = F->region[best];
        const double* n = F->geom + 11 * best;
        s0 = (E.x * n[0] + E.y * n[1] + E.z * n[2]) >= 0.0 ? 1.0 : -1.0;
    } else {
        s0 = (dot(E, x) >= 0.0) ? 1.0 : -1.0;
    }
    int side = norm(E) > P->E0 ? 1 : -1;
    int st = 3;
    int64_t step = 0;
    for (; step < P->max_steps; ++step) {
        field_pt(F, x, seed_region, &E, &ind);
        if (!isfinite(norm(E))) { st = -1; break; }  /* on an edge or vertex: singular field */
        if (norm(E) < P->e_floor) { st = 4; break; }
        double rem = P->h;
        int done = 0;
        for (int nev = 0; rem > 0.0 && nev < 4; ++nev) {
            vec x1;
            double K1;
            rk4_step(F, P, seed_region, s0, side, x, K, rem, &x1, &K1);
            vec E1;
            double ind1;
            field_pt(F, x1, seed_region, &E1, &ind1);
            double best = 2.0 * rem;
            int which = -1;
            if ((norm(E1) > P->E0) != (side > 0)) {
                double ga = event_g(F, P, seed_region, s0, side, x, K, 0.0, EV_ALPHA);
                double sg = illinois(F, P, seed_region, s0, side, x, K, rem, ga, norm(E1) - P->E0, EV_ALPHA);
                if (sg < best) { best = sg; which = EV_ALPHA; }
            }
            if (norm(x1) >= P->r_max) {
                double sg = illinois(F, P, seed_region, s0, side, x, K, rem, norm(x) - P->r_max,
                                     norm(x1) - P->r_max, EV_RMAX);
                if (sg < best) { best = sg; which = EV_RMAX; }
            }
            if (ind1 < -0.5) {
                double ga = event_g(F, P, seed_region, s0, side, x, K, 0.0, EV_ELECTRODE);
                double sg = illinois(F, P, seed_region, s0, side, x, K, rem, ga, ind1 + 0.5, EV_ELECTRODE);
                if (sg < best) { best = sg; which = EV_ELECTRODE; }
            }
            if (which < 0) {
                x = x1; K = K1; rem = 0.0;
                break;
            }
            rk4_step(F, P, seed_region, s0, side, x, K, best, &x, &K);
            if (which == EV_ALPHA) {
                side = -side;
                rem -= best;
                continue;
            }
            st = which == EV_RMAX ? 1 : 2;
            done = 1;
            break;
        }
        if (done) break;
    }
    *K_out = K;
    *status = st;
    *nsteps = (int32_t)step;
    xend[0] = x.x; xend[1] = x.y; xend[2] = x.z;
}

/* L field lines from seeds[L][3].  analytic != 0: point-charge field of strength q
 * (mesh arguments unused).  electrode[nregions]: 1 for conductor/floating regions. */
void oracle_trace(int64_t L, const double* seeds, int analytic, double q, int64_t np,
                  const double* X, const int32_t* tri, const double* geom, const double* u,
                  const int32_t* region, const int32_t* electrode, double eta, int nu,
                  const double* uk, const double* wu, int nv, const double* vl, const double* wv,
                  double h, double r_max, double c, double E0, double d, double e_floor,
                  int64_t max_steps, double* K, int32_t* status, int32_t* nsteps, double* xend)
{
    fsrc F = {analytic, q, np, X, tri, geom, u, region, electrode, eta, nu, nv, uk, wu, vl, wv};
    tparams P = {h, r_max, c, E0, d, e_floor, max_steps};
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t l = 0; l < L; ++l)
        trace_one(&F, &P, seeds + 3 * l, K + l, status + l, nsteps + l, xend + 3 * l);
}

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
 *   oracle_set_threads      OpenMP thread count of the loops above (timing only)
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct { double x, y, z; } vec;

/* Set the OpenMP thread count of the oracle's parallel loops; returns the count
 * in force before.  n <= 0 leaves it unchanged. */
int oracle_set_threads(int n)
{
    const int before = omp_get_max_threads();
    if (n > 0) omp_set_num_threads(n);
    return before;
}

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

/* Sub-steps of one traced line, recorded for the reverse pass (oracle adjoint).
 * dep: how the sub-step's length s depends on the data:
 *   0: constant (a full first sub-step of length h, or an event located at 0);
 *   1: s = what remains of the step, h minus the earlier sub-steps of the same step;
 *   2: s is a located root of the event function ev (implicit in x and the field). */
typedef struct { vec x; double K, s; int side, dep, ev, first; } sstep;
typedef struct { sstep* v; int64_t n, cap; } tape_t;

static void tape_push(tape_t* t, vec x, double K, double s, int side, int dep, int ev, int first)
{
    if (!t) return;
    if (t->n == t->cap) {
        t->cap = t->cap ? 2 * t->cap : 1024;
        t->v = (sstep*)realloc(t->v, (size_t)t->cap * sizeof(sstep));
    }
    sstep e = {x, K, s, side, dep, ev, first};
    t->v[t->n++] = e;
}

static void trace_one(const fsrc* F, const tparams* P, const double* seed, double* K_out,
                      int32_t* status, int32_t* nsteps, double* xend, tape_t* tape, double* s0_out,
                      int* seed_region_out)
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
            const int first = nev == 0, dep_rem = nev == 0 ? 0 : 1;
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
                tape_push(tape, x, K, rem, side, dep_rem, -1, first);
                x = x1; K = K1; rem = 0.0;
                break;
            }
            tape_push(tape, x, K, best, side, best == 0.0 ? 0 : (best == rem ? dep_rem : 2), which, first);
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
    if (s0_out) *s0_out = s0;
    if (seed_region_out) *seed_region_out = seed_region;
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
        trace_one(&F, &P, seeds + 3 * l, K + l, status + l, nsteps + l, xend + 3 * l, NULL, NULL, NULL);
}

/* ================================================================ adjoint */
/*
 * Gradient of J = sum_l w_l K_l (Eq. Breakdowncrit along each line) by a hand-written
 * reverse pass over exactly the steps trace_one takes.  The paper has no adjoint;
 * this is the plain FP64 reference the GPU adjoint is checked against.
 *
 * Forward map of one sub-step of length s from x on branch `side` (classical RK4 on
 * dx/ds = f(x) = s0 E(x)/|E(x)|, dK/ds = alpha(|E(x)|)):
 *   y1 = x, y2 = x + s/2 k1, y3 = x + s/2 k2, y4 = x + s k3,  k_i = f(y_i),
 *   x1 = x + s/6 (k1 + 2 k2 + 2 k3 + k4),  K1 = K + s/6 (a1 + 2 a2 + 2 a3 + a4).
 * Reverse: with adjoints lx1 (of x1) and lK (of K, constant w_l), the stage adjoints are
 * lk_i = s c_i/6 lx1 and la_i = s c_i/6 lK (c = 1, 2, 2, 1), taken back through the
 * stages in reverse order:
 *   lE_i = s0/|E| (I - e e^T) lk_i + alpha'(|E|) e la_i        (e = E/|E| at y_i)
 *   ly_i = (dE/dy)^T lE_i;   lx += ly_i;   lk_{i-1} += c'_i s ly_i;   ls += c'_i k_{i-1}.ly_i
 * and every lE_i is also applied to the explicit dependence of E(y_i) = sum_j u_j G_j(y_i)
 * on the density (dJ/du_j += lE.G_j) and on the panel vertices (u_j lE.dG_j/dX).
 * A sub-step whose length is a located event root (|E(x1)| = E0 or |x1| = r_max)
 * carries the implicit-function term: with g(x1) the event function and
 * v = dg/dx1, the root moves by  ds = -(v.dx1 + dg_explicit) / (v.dx1/ds),  so the
 * adjoint ls of the length is sent back as an adjoint -ls/(v.dx1/ds) on x1 through the
 * same sub-step at fixed s (plus, for |E| = E0, on the field at x1).  A sub-step that
 * ends a step takes what remains of h; its ls goes to the earlier lengths with a minus.
 *
 * Pair derivatives: regular pairs (D > eta R) are differentiated on their nodes,
 * y_k = a + u (b-a) + u v (c-b) with barycentric weights (1-u, u(1-v), uv) and
 * weights w_k = 2A uhat_k; d(2A)/dv_i = n x (v_{i+2} - v_{i+1}).  Near pairs take the
 * closed form of oracle_tri_exact evaluated in complex arithmetic with one input
 * shifted by i*1e-30 (complex-step differentiation, Squire & Trapp 1998): the
 * imaginary part over 1e-30 is the derivative to rounding.
 */
#include <complex.h>

typedef struct { double complex x, y, z; } cvec;
static cvec csub(cvec a, cvec b) { cvec r = {a.x - b.x, a.y - b.y, a.z - b.z}; return r; }
static cvec cadd(cvec a, cvec b) { cvec r = {a.x + b.x, a.y + b.y, a.z + b.z}; return r; }
static cvec cscl(cvec a, double complex s) { cvec r = {a.x * s, a.y * s, a.z * s}; return r; }
static double complex cdot(cvec a, cvec b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static cvec ccross(cvec a, cvec b)
{
    cvec r = {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
    return r;
}
static double complex cnorm(cvec a) { return csqrt(cdot(a, a)); }

/* atan2 continued to numbers with an infinitesimal imaginary part (first order) */
static double complex cs_atan2(double complex y, double complex x)
{
    const double yr = creal(y), xr = creal(x);
    return atan2(yr, xr) + I * (xr * cimag(y) - yr * cimag(x)) / (xr * xr + yr * yr);
}

/* oracle_tri_exact in complex arithmetic (same formulas; branches by real parts) */
static void tri_exact_cx(cvec x, cvec v0, cvec v1, cvec v2, int self, double complex* S,
                         cvec* G)
{
    cvec v[3] = {v0, v1, v2};
    cvec w = ccross(csub(v[1], v[0]), csub(v[2], v[0]));
    cvec n = cscl(w, 1.0 / cnorm(w));
    double complex h = cdot(csub(x, v[0]), n);
    double complex sum_df = 0.0;
    cvec gin = {0.0, 0.0, 0.0};
    for (int i = 0; i < 3; ++i) {
        cvec p0 = v[i], p1 = v[(i + 1) % 3];
        cvec e = csub(p1, p0);
        cvec t = cscl(e, 1.0 / cnorm(e));
        cvec m = ccross(t, n);
        double complex s0 = cdot(csub(p0, x), t), s1 = cdot(csub(p1, x), t);
        double complex r0 = cnorm(csub(p0, x)), r1 = cnorm(csub(p1, x));
        double complex d = cdot(csub(p0, x), m);
        double complex f;
        if (creal(s0) >= 0.0)
            f = clog((r1 + s1) / (r0 + s0));
        else if (creal(s1) <= 0.0)
            f = clog((r0 - s0) / (r1 - s1));
        else
            f = clog((r1 + s1) * (r0 - s0) / (d * d + h * h));
        /* d f is 0 where d is; its derivative f d' is not, unless x lies on the edge
         * itself (f infinite: the field is singular there) */
        if (isfinite(creal(f))) sum_df += d * f;
        gin = cadd(gin, cscl(m, f));
    }
    double complex omega = 0.0;
    if (!self) {
        cvec A0 = csub(v[0], x), A1 = csub(v[1], x), A2 = csub(v[2], x);
        double complex l0 = cnorm(A0), l1 = cnorm(A1), l2 = cnorm(A2);
        double complex num = cdot(A0, ccross(A1, A2));
        double complex den = l0 * l1 * l2 + cdot(A0, A1) * l2 + cdot(A0, A2) * l1 + cdot(A1, A2) * l0;
        omega = 2.0 * cs_atan2(num, den);
    }
    const double k = 1.0 / (4.0 * M_PI);
    *S = k * (sum_df + h * omega);
    cvec g = csub(gin, cscl(n, omega));
    *G = cscl(g, k);
}

static const double kCS = 1e-30;

/* Derivatives of the closed form by complex step.  Inputs q = 0..11: x (0..2), a, b, c.
 * Outputs dS[q], dG[q][3].  centroid != 0: x is the centroid of (a, b, c) and moves with
 * them (then q < 3 is not used); self marks x as the panel's own centroid. */
static void tri_exact_derivs(vec x, vec a, vec b, vec c, int self, int centroid, double dS[12],
                             double dG[12][3])
{
    for (int q = centroid ? 3 : 0; q < 12; ++q) {
        double in[12] = {x.x, x.y, x.z, a.x, a.y, a.z, b.x, b.y, b.z, c.x, c.y, c.z};
        double complex z[12];
        for (int k = 0; k < 12; ++k) z[k] = in[k];
        z[q] += I * kCS;
        cvec cx = {z[0], z[1], z[2]}, ca = {z[3], z[4], z[5]}, cb = {z[6], z[7], z[8]},
             cc = {z[9], z[10], z[11]};
        if (centroid) cx = cscl(cadd(cadd(ca, cb), cc), 1.0 / 3.0);
        double complex S;
        cvec G;
        tri_exact_cx(cx, ca, cb, cc, self, &S, &G);
        dS[q] = cimag(S) / kCS;
        dG[q][0] = cimag(G.x) / kCS;
        dG[q][1] = cimag(G.y) / kCS;
        dG[q][2] = cimag(G.z) / kCS;
    }
    if (centroid)
        for (int k = 0; k < 3; ++k) {
            dS[k] = 0.0;
            dG[k][0] = dG[k][1] = dG[k][2] = 0.0;
        }
}

/* d(2A)/dv_i = n x (v_{i+2} - v_{i+1}) for the three vertices */
static void darea2(vec v[3], vec n, vec out[3])
{
    for (int i = 0; i < 3; ++i) out[i] = cross(n, sub(v[(i + 2) % 3], v[(i + 1) % 3]));
}

/* Per-thread accumulators of the reverse pass. */
typedef struct {
    double* gu;   /* [np] dJ/du_j */
    double* gX;   /* [nv][3] explicit vertex derivative */
    double gq;    /* analytic field: dJ/dq */
} adj_acc;

/* vertices of panel j */
static void panel_vertices(const fsrc* F, int64_t j, vec v[3])
{
    for (int i = 0; i < 3; ++i) v[i] = mk(F->X + 3 * (int64_t)F->tri[3 * j + i]);
}

/* E(y), its Jacobian J = dE/dy (row-major 3x3), and -- if lam != NULL -- the explicit
 * derivative of lam.E(y) with respect to the density and the panel vertices, added to
 * acc.  Same pair classification as field_pt. */
static void field_adj(const fsrc* F, vec y, const vec* lam, vec* E, double J[9], adj_acc* acc)
{
    for (int k = 0; k < 9; ++k) J[k] = 0.0;
    if (F->analytic) {
        double r = norm(y), r3 = r * r * r, r5 = r3 * r * r;
        *E = scl(y, F->q / r3);
        double yy[3] = {y.x, y.y, y.z};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                J[3 * a + b] = F->q * ((a == b ? 1.0 / r3 : 0.0) - 3.0 * yy[a] * yy[b] / r5);
        if (lam && acc) acc->gq += dot(*lam, scl(y, 1.0 / r3));
        return;
    }
    const double kk = 1.0 / (4.0 * M_PI);
    vec e = {0.0, 0.0, 0.0};
    for (int64_t j = 0; j < F->np; ++j) {
        const double* g = F->geom + 11 * j;
        const double uj = F->u[j];
        vec v[3];
        panel_vertices(F, j, v);
        double dx = y.x - g[7], dy = y.y - g[8], dz = y.z - g[9];
        int regular = sqrt(dx * dx + dy * dy + dz * dz) > F->eta * g[10];
        if (regular) {
            vec ab = sub(v[1], v[0]), bc = sub(v[2], v[1]);
            double A2 = norm(cross(ab, sub(v[2], v[0])));
            vec Gs = {0.0, 0.0, 0.0};
            double sA = 0.0;           /* sum_k uhat_k lam.d/r^3 (area part) */
            vec gv[3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
            for (int k = 0; k < F->nu; ++k)
                for (int l = 0; l < F->nv; ++l) {
                    double uu = F->uk[k], vv = F->vl[l];
                    double wh = uu * F->wu[k] * F->wv[l];
                    double w = A2 * wh;
                    vec yk = add(v[0], add(scl(ab, uu), scl(bc, uu * vv)));
                    vec d = sub(y, yk);
                    double r2 = dot(d, d), r = sqrt(r2), ir3 = 1.0 / (r2 * r);
                    Gs = add(Gs, scl(d, w * ir3));
                    double dd[3] = {d.x, d.y, d.z};
                    double H[9];
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b)
                            H[3 * a + b] = ir3 * ((a == b ? 1.0 : 0.0) - 3.0 * dd[a] * dd[b] / r2);
                    for (int q = 0; q < 9; ++q) J[q] += kk * uj * w * H[q];
                    if (lam && acc) {
                        vec t = {H[0] * lam->x + H[1] * lam->y + H[2] * lam->z,
                                 H[3] * lam->x + H[4] * lam->y + H[5] * lam->z,
                                 H[6] * lam->x + H[7] * lam->y + H[8] * lam->z};
                        double bw[3] = {1.0 - uu, uu * (1.0 - vv), uu * vv};
                        for (int a = 0; a < 3; ++a) gv[a] = add(gv[a], scl(t, -w * bw[a]));
                        sA += wh * dot(*lam, d) * ir3;
                    }
                }
            e = add(e, scl(Gs, kk * uj));
            if (lam && acc) {
                acc->gu[j] += kk * dot(*lam, Gs);
                vec n = {g[0], g[1], g[2]}, dA[3];
                darea2(v, n, dA);
                for (int a = 0; a < 3; ++a) {
                    vec tot = scl(add(gv[a], scl(dA[a], sA)), kk * uj);
                    double* o = acc->gX + 3 * (int64_t)F->tri[3 * j + a];
                    o[0] += tot.x; o[1] += tot.y; o[2] += tot.z;
                }
            }
        } else {
            double s, gg[3], yp[3] = {y.x, y.y, y.z};
            oracle_tri_exact(yp, F->X + 3 * (int64_t)F->tri[3 * j], F->X + 3 * (int64_t)F->tri[3 * j + 1],
                             F->X + 3 * (int64_t)F->tri[3 * j + 2], 0, &s, gg);
            vec Gj = {gg[0], gg[1], gg[2]};
            e = add(e, scl(Gj, uj));
            double dS[12], dG[12][3];
            tri_exact_derivs(y, v[0], v[1], v[2], 0, 0, dS, dG);
            for (int b = 0; b < 3; ++b)
                for (int a = 0; a < 3; ++a) J[3 * a + b] += uj * dG[b][a];   /* column b: d/dy_b */
            if (lam && acc) {
                acc->gu[j] += dot(*lam, Gj);
                for (int a = 0; a < 3; ++a) {
                    double* o = acc->gX + 3 * (int64_t)F->tri[3 * j + a];
                    for (int c = 0; c < 3; ++c) {
                        const double* dg = dG[3 + 3 * a + c];
                        o[c] += uj * (lam->x * dg[0] + lam->y * dg[1] + lam->z * dg[2]);
                    }
                }
            }
        }
    }
    *E = e;
}

static double alpha_prime(const tparams* P, double Em, int side)
{
    return side > 0 ? 2.0 * P->c * (Em - P->E0) : 0.0;
}

static vec matTvec(const double J[9], vec l)
{
    vec r = {J[0] * l.x + J[3] * l.y + J[6] * l.z, J[1] * l.x + J[4] * l.y + J[7] * l.z,
             J[2] * l.x + J[5] * l.y + J[8] * l.z};
    return r;
}

static vec matvec3(const double J[9], vec l)
{
    vec r = {J[0] * l.x + J[1] * l.y + J[2] * l.z, J[3] * l.x + J[4] * l.y + J[5] * l.z,
             J[6] * l.x + J[7] * l.y + J[8] * l.z};
    return r;
}

/* The four stage points y_i and slopes k_i of an RK4 sub-step of length s from x. */
static void rk4_stages(const fsrc* F, double s0, vec x, double s, vec y[4], vec k[4], vec E[4])
{
    double J[9];
    for (int st = 0; st < 4; ++st) {
        y[st] = st == 0 ? x : add(x, scl(k[st - 1], st < 3 ? 0.5 * s : s));
        field_adj(F, y[st], NULL, &E[st], J, NULL);
        k[st] = scl(E[st], s0 / norm(E[st]));
    }
}

/* Reverse of one RK4 sub-step at fixed length s: given the adjoint lx1 of its end
 * point and lK of K, add to *lx the adjoint of its start point and to acc the explicit
 * derivatives; return the adjoint of the length s. */
static double rk4_reverse(const fsrc* F, const tparams* P, double s0, int side, vec x, double s,
                          vec lx1, double lK, vec* lx, adj_acc* acc)
{
    static const double cw[4] = {1.0, 2.0, 2.0, 1.0};
    static const double cy[4] = {0.0, 0.5, 0.5, 1.0};   /* y_i = x + cy_i s k_{i-1} */
    vec y[4], k[4], E[4];
    rk4_stages(F, s0, x, s, y, k, E);
    vec lk[4];
    double ls = 0.0;
    for (int st = 0; st < 4; ++st) {
        lk[st] = scl(lx1, s * cw[st] / 6.0);
        ls += cw[st] / 6.0 * (dot(lx1, k[st]) + lK * alpha_eff(P, norm(E[st]), side));
    }
    vec lxs = lx1;
    for (int st = 3; st >= 0; --st) {
        const double Em = norm(E[st]);
        vec e = scl(E[st], 1.0 / Em);
        vec lE = scl(sub(lk[st], scl(e, dot(e, lk[st]))), s0 / Em);
        lE = add(lE, scl(e, alpha_prime(P, Em, side) * lK * s * cw[st] / 6.0));
        vec Ed;
        double J[9];
        field_adj(F, y[st], &lE, &Ed, J, acc);
        vec ly = matTvec(J, lE);
        lxs = add(lxs, ly);
        if (st > 0) {
            lk[st - 1] = add(lk[st - 1], scl(ly, cy[st] * s));
            ls += cy[st] * dot(k[st - 1], ly);
        }
    }
    *lx = add(*lx, lxs);
    return ls;
}

/* d x1 / d s of an RK4 sub-step of length s from x (forward tangent in s). */
static vec rk4_dsigma(const fsrc* F, double s0, vec x, double s)
{
    static const double cw[4] = {1.0, 2.0, 2.0, 1.0};
    static const double cy[4] = {0.0, 0.5, 0.5, 1.0};
    vec y = x, k[4], dk[4], dy = {0.0, 0.0, 0.0};
    vec out = {0.0, 0.0, 0.0};
    for (int st = 0; st < 4; ++st) {
        if (st > 0) {
            y = add(x, scl(k[st - 1], cy[st] * s));
            dy = add(scl(k[st - 1], cy[st]), scl(dk[st - 1], cy[st] * s));
        }
        vec E;
        double J[9];
        field_adj(F, y, NULL, &E, J, NULL);
        const double Em = norm(E);
        vec e = scl(E, 1.0 / Em);
        k[st] = scl(E, s0 / Em);
        vec dE = matvec3(J, dy);
        dk[st] = scl(sub(dE, scl(e, dot(e, dE))), s0 / Em);
        out = add(out, add(scl(k[st], cw[st] / 6.0), scl(dk[st], s * cw[st] / 6.0)));
    }
    return out;
}

/* Implicit-function term of a sub-step whose length s is a located root of event ev:
 * the adjoint ls of s becomes adjoints of the start point and the field. */
static void event_reverse(const fsrc* F, const tparams* P, double s0, int side, vec x, double s,
                          int ev, double ls, vec* lx, adj_acc* acc)
{
    if (ls == 0.0) return;
    vec x1;
    double K1;
    rk4_step(F, P, -1, s0, side, x, 0.0, s, &x1, &K1);
    vec dx1 = rk4_dsigma(F, s0, x, s);
    vec v;
    vec E1, e1 = {0.0, 0.0, 0.0};
    double J1[9];
    if (ev == EV_RMAX) {
        v = scl(x1, 1.0 / norm(x1));
    } else {
        field_adj(F, x1, NULL, &E1, J1, NULL);
        e1 = scl(E1, 1.0 / norm(E1));
        v = matTvec(J1, e1);
    }
    const double mu = -ls / dot(v, dx1);
    rk4_reverse(F, P, s0, side, x, s, scl(v, mu), 0.0, lx, acc);
    if (ev == EV_ALPHA) {
        vec lE = scl(e1, mu), Ed;
        double Jd[9];
        field_adj(F, x1, &lE, &Ed, Jd, acc);
    }
}

/* Reverse pass of one traced line with weight wl: adds dJ/du and the explicit vertex
 * derivative (and dJ/dq for the analytic field) to acc. */
static void line_reverse(const fsrc* F, const tparams* P, double s0, const tape_t* tp, double wl,
                         adj_acc* acc)
{
    vec lx = {0.0, 0.0, 0.0};      /* the end point does not enter J */
    double pend = 0.0;             /* adjoint owed to the earlier lengths of the step */
    for (int64_t t = tp->n - 1; t >= 0; --t) {
        const sstep* ss = tp->v + t;
        vec lx_start = {0.0, 0.0, 0.0};
        double ls = 0.0;
        if (ss->s > 0.0) ls = rk4_reverse(F, P, s0, ss->side, ss->x, ss->s, lx, wl, &lx_start, acc);
        else lx_start = lx;
        if (ss->dep == 1) {
            pend = -ls;            /* s = h - (earlier lengths of this step) */
        } else if (ss->dep == 2) {
            event_reverse(F, P, s0, ss->side, ss->x, ss->s, ss->ev, ls + pend, &lx_start, acc);
        }
        lx = lx_start;
        if (ss->first) pend = 0.0;
    }
}

/* Adjoint of L field lines (arguments as oracle_trace; w[L] the weights w_l of J):
 * K, status per line; gu[np] = dJ/du (explicit, through the field along the lines);
 * gX[nv][3] = explicit dJ/dX through the panel geometry of those fields; *gq = dJ/dq
 * for the analytic field.  Returns -1 (and no gradient) if a line ended on another
 * electrode or at a singular field (status 2 or -1), else 0. */
int oracle_adjoint_trace(int64_t L, const double* seeds, int analytic, double q, int64_t np,
                         int64_t nvert, const double* X, const int32_t* tri, const double* geom,
                         const double* u, const int32_t* region, const int32_t* electrode,
                         double eta, int nu, const double* uk, const double* wu, int nv,
                         const double* vl, const double* wv, double h, double r_max, double c,
                         double E0, double d, double e_floor, int64_t max_steps, const double* w,
                         double* K, int32_t* status, double* gu, double* gX, double* gq)
{
    fsrc F = {analytic, q, np, X, tri, geom, u, region, electrode, eta, nu, nv, uk, wu, vl, wv};
    tparams P = {h, r_max, c, E0, d, e_floor, max_steps};
    int bad = 0;
    for (int64_t j = 0; j < np; ++j) gu[j] = 0.0;
    for (int64_t k = 0; k < 3 * nvert; ++k) gX[k] = 0.0;
    *gq = 0.0;
#pragma omp parallel
    {
        adj_acc acc;
        acc.gu = (double*)calloc((size_t)(np > 0 ? np : 1), sizeof(double));
        acc.gX = (double*)calloc((size_t)(nvert > 0 ? 3 * nvert : 1), sizeof(double));
        acc.gq = 0.0;
#pragma omp for schedule(dynamic, 1)
        for (int64_t l = 0; l < L; ++l) {
            tape_t tp = {NULL, 0, 0};
            double s0 = 1.0, xe[3];
            int32_t ns;
            int sr;
            trace_one(&F, &P, seeds + 3 * l, K + l, status + l, &ns, xe, &tp, &s0, &sr);
            if (status[l] == 2 || status[l] == -1) {
#pragma omp atomic write
                bad = 1;
            } else {
                line_reverse(&F, &P, s0, &tp, w[l], &acc);
            }
            free(tp.v);
        }
#pragma omp critical
        {
            for (int64_t j = 0; j < np; ++j) gu[j] += acc.gu[j];
            for (int64_t k = 0; k < 3 * nvert; ++k) gX[k] += acc.gX[k];
            *gq += acc.gq;
        }
        free(acc.gu);
        free(acc.gX);
    }
    return bad ? -1 : 0;
}

/* Collocation part of the adjoint: gX[nv][3] += d/dX of
 *     sum_i sum_j u_j (alpha_i S_j(c_i) + beta_i n_i . G_j(c_i))
 * with the pair integrals of the method (mode 1) and c_i the centroid of triangle i,
 * which moves with its vertices; n_i is held fixed here (its variation is applied by
 * the caller).  For the self pair (j = i) the normal part of G is the principal value
 * 0 for every shape, so only alpha_i S_ii enters, differentiated with the centroid
 * moving. */
void oracle_adjoint_rows(int64_t np, int64_t nvert, const double* X, const int32_t* tri,
                         const double* geom, const double* u, const double* alpha, const double* beta,
                         double eta, int nu, const double* uk, const double* wu, int nv,
                         const double* vl, const double* wv, double* gX)
{
    const double kk = 1.0 / (4.0 * M_PI);
    for (int64_t k = 0; k < 3 * nvert; ++k) gX[k] = 0.0;
#pragma omp parallel
    {
        double* acc = (double*)calloc((size_t)(3 * nvert), sizeof(double));
#pragma omp for schedule(dynamic, 4)
        for (int64_t i = 0; i < np; ++i) {
            if (alpha[i] == 0.0 && beta[i] == 0.0) continue;
            const double* gi = geom + 11 * i;
            vec x = {gi[4], gi[5], gi[6]}, ni = {gi[0], gi[1], gi[2]};
            vec gx = {0.0, 0.0, 0.0};   /* derivative with respect to the target c_i */
            for (int64_t j = 0; j < np; ++j) {
                const double* g = geom + 11 * j;
                const double uj = u[j];
                vec v[3];
                for (int a = 0; a < 3; ++a) v[a] = mk(X + 3 * (int64_t)tri[3 * j + a]);
                double gv[3][3] = {{0}};
                if (j == i) {
                    double dS[12], dG[12][3];
                    tri_exact_derivs(x, v[0], v[1], v[2], 1, 1, dS, dG);
                    for (int a = 0; a < 3; ++a)
                        for (int c = 0; c < 3; ++c) gv[a][c] = alpha[i] * uj * dS[3 + 3 * a + c];
                } else {
                    double dx = x.x - g[7], dy = x.y - g[8], dz = x.z - g[9];
                    int regular = sqrt(dx * dx + dy * dy + dz * dz) > eta * g[10];
                    if (regular) {
                        vec ab = sub(v[1], v[0]), bc = sub(v[2], v[1]);
                        double A2 = norm(cross(ab, sub(v[2], v[0])));
                        double sS = 0.0, sG = 0.0;     /* area parts */
                        vec nodev[3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
                        for (int k = 0; k < nu; ++k)
                            for (int l = 0; l < nv; ++l) {
                                double uu = uk[k], vv = vl[l];
                                double wh = uu * wu[k] * wv[l], w = A2 * wh;
                                vec yk = add(v[0], add(scl(ab, uu), scl(bc, uu * vv)));
                                vec d = sub(x, yk);
                                double r2 = dot(d, d), r = sqrt(r2), ir3 = 1.0 / (r2 * r);
                                double dn = dot(d, ni);
                                /* H n = ir3 (n - 3 d (d.n)/r^2) */
                                vec Hn = scl(sub(ni, scl(d, 3.0 * dn / r2)), ir3);
                                /* d/dy_k of alpha S + beta n.G:  alpha w d/r^3 - beta w H n */
                                vec gy = sub(scl(d, alpha[i] * w * ir3), scl(Hn, beta[i] * w));
                                gx = sub(gx, scl(gy, kk * uj));   /* d/dx = -d/dy */
                                double bw[3] = {1.0 - uu, uu * (1.0 - vv), uu * vv};
                                for (int a = 0; a < 3; ++a) nodev[a] = add(nodev[a], scl(gy, bw[a]));
                                sS += wh / r;
                                sG += wh * dn * ir3;
                            }
                        vec nj = {g[0], g[1], g[2]}, dA[3];
                        darea2(v, nj, dA);
                        for (int a = 0; a < 3; ++a) {
                            vec t = scl(add(nodev[a], scl(dA[a], alpha[i] * sS + beta[i] * sG)), kk * uj);
                            gv[a][0] = t.x; gv[a][1] = t.y; gv[a][2] = t.z;
                        }
                    } else {
                        double dS[12], dG[12][3];
                        tri_exact_derivs(x, v[0], v[1], v[2], 0, 0, dS, dG);
                        double q[12];
                        for (int m = 0; m < 12; ++m)
                            q[m] = uj * (alpha[i] * dS[m] + beta[i] * (ni.x * dG[m][0] + ni.y * dG[m][1] +
                                                                         ni.z * dG[m][2]));
                        gx.x += q[0]; gx.y += q[1]; gx.z += q[2];
                        for (int a = 0; a < 3; ++a)
                            for (int c = 0; c < 3; ++c) gv[a][c] = q[3 + 3 * a + c];
                    }
                }
                for (int a = 0; a < 3; ++a) {
                    double* o = acc + 3 * (int64_t)tri[3 * j + a];
                    o[0] += gv[a][0]; o[1] += gv[a][1]; o[2] += gv[a][2];
                }
            }
            /* the target is the centroid: a third to each vertex of triangle i */
            for (int a = 0; a < 3; ++a) {
                double* o = acc + 3 * (int64_t)tri[3 * i + a];
                o[0] += gx.x / 3.0; o[1] += gx.y / 3.0; o[2] += gx.z / 3.0;
            }
        }
#pragma omp critical
        for (int64_t k = 0; k < 3 * nvert; ++k) gX[k] += acc[k];
        free(acc);
    }
}

/* Public entry of the complex-step pair derivatives (for tests): dS[12], dG[12][3]
 * with respect to x, a, b, c (see tri_exact_derivs). */
void oracle_tri_exact_derivs(const double* xp, const double* ap, const double* bp, const double* cp,
                             int self, int centroid, double* dS, double* dG)
{
    double gg[12][3];
    tri_exact_derivs(mk(xp), mk(ap), mk(bp), mk(cp), self, centroid, dS, gg);
    for (int q = 0; q < 12; ++q)
        for (int k = 0; k < 3; ++k) dG[3 * q + k] = gg[q][k];
}

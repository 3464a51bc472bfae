// p1.cu -- the paper's own discretisation on the GPU: mapped linear (P1) basis
// functions on curved quadratic (six-node) triangles, collocated at the vertices
// (Sec. 3), with the pair types of Sec. 4 for (collocation point, triangle):
//   singular       the point is a corner of the triangle: a Duffy rule collapsed at
//                  that corner;
//   regular        D > eta R (D the distance to the circumcentre of the three
//                  corners, R their circumradius): a Duffy rule collapsed at corner
//                  0, g x g Gauss-Legendre points in (s, t);
//   near-singular  otherwise: the triangle is split at its point closest to x
//                  (projected Gauss-Newton on the quadratic map) into the parts
//                  that have that point as a corner, each collapsed there, the
//                  radial variable refined geometrically toward it down to a tenth
//                  of distance / size.
// Eq. Matrix: v_ij = sum_T int psi_j(y) / (4 pi |x_i - y|) dS_y, psi_j the mapped
// linear function of vertex j.
//
// GPU design.  The regular pairs run through the same regular-pair kernels as the
// flat panels: each curved triangle contributes its g x g rule points y_q with the
// density folded into the weight, w_q J_q sigma_h(y_q) = w_q J_q sum_k lambda_k(q)
// u_{v_k}, refolded per product by one kernel.  The singular and near-singular
// integrals do not depend on the density: they are computed once at set-up in
// FP64 (one warp per (vertex, triangle) pair) and kept in a CSR over the vertices
// with three values per pair, one per corner's basis function.  A product's row
// kernel gives every collocation point its own warp (the paper's collision-free
// row ownership: a row is written by one owner only).  Dense rows are assembled
// with one thread per collocation point looping over all triangles.
//
// Row equations: conductor vertices sum_j v_ij u_j = V0 (Eq. Final1); floating
// vertices sum_j v_ij u_j - V_f = 0 (Eq. Final2); the neutrality row of a closed
// floating body in the form Gauss's law gives it, int_body sigma_h dS = 0 (Eq.
// Final4 with no field inside a conductor); dielectric vertices
// (eps+ + eps-)/2 u_i + (eps+ - eps-) (K'u)_i = 0 (Eq. Final3), where K'u at a vertex
// of a C0 mesh of curved triangles is taken through the jump relations (Eq. ADL) as
// Plemelj's formulas: the mean of the two one-sided normal fields, each the field at
// x_i +- delta n_i extrapolated to delta -> 0 from delta and 2 delta (delta = 1e-3 of
// the mean edge at x_i; n_i the normalised sum of the adjacent triangles' normals at
// that corner).  The regular pairs of those four points go through the far kernel
// every product; their near pairs' normal fields are computed once at set-up (CSR).
// Sheets are not built on this path.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "bem_internal.cuh"

struct P1Data {
    int64_t nn = 0, nv = 0, N = 0;
    int g = 4, Q = 16;
    int sing_n = 24, near_n = 16, near_nt = 64;
    double* nodes = nullptr;       // [nn][3]
    int32_t* tri6 = nullptr;       // [N][6]
    double* lam = nullptr;         // [Q][3] basis values at the regular rule's points
    double* rule = nullptr;        // [2 g] Gauss-Legendre points and weights on [0, 1]
    double* sing_rule = nullptr;   // [2 sing_n]
    double* near_rule = nullptr;   // [2 near_n]
    double* near_trule = nullptr;  // [2 near_nt]
    int64_t nnz = 0;
    int64_t* ptr = nullptr;        // [nv+1] near pairs of every vertex, triangles ascending
    int32_t* col = nullptr;        // [nnz] triangle
    uint8_t* flag = nullptr;       // [nnz] bit0: near in FP32, bit1: in FP64, bit2: singular
    double* val = nullptr;         // [nnz][3] singular / near-singular basis integrals (with 1/4pi)
    double* neut_w = nullptr;      // [nfloat][nv] int psi_v over each floating body
    int32_t* vkind = nullptr;      // [nv] row kind (BEM_CONDUCTOR or BEM_FLOATING)
    int32_t* vaux = nullptr;       // [nv] region of a conductor vertex, floating id
    int32_t* phi_all = nullptr;    // [nv] BEM_CONDUCTOR: every row needs phi alone
    double* ones = nullptr;        // [N] density factor of the folded FP64 kernel
    int32_t* d_region = nullptr;   // [N]
    // dielectric rows (Eq. Final3): K'u at a vertex as the mean of the two one-sided
    // normal fields, each the field at x_i +- m delta_i n_i (m = 1, 2) extrapolated to
    // delta -> 0; the four points of dielectric vertex d are 4d .. 4d+3
    int64_t nd = 0;                // dielectric vertices
    int32_t* dvert = nullptr;      // [nd] their vertex indices
    int32_t* didx = nullptr;       // [nv] index of a vertex among them, -1 for other vertices
    double* dpts = nullptr;        // [4 nd][3] x + delta n, x - delta n, x + 2 delta n, x - 2 delta n
    double* dnrm = nullptr;        // [nd][3] vertex normal n_i
    double* dcoef = nullptr;       // [nv][2] (eps+ + eps-)/2 and eps+ - eps- of a dielectric vertex
    int64_t dnnz = 0;
    int64_t* dptr = nullptr;       // [4 nd + 1] near pairs of every point, triangles ascending
    int32_t* dcol = nullptr;       // [dnnz]
    uint8_t* dflag = nullptr;      // [dnnz] bit0: near in FP32, bit1: in FP64
    double* dval = nullptr;        // [dnnz][3] c_m (G_k . n_i) of the near-singular integrals
};

// weight of point k (0..3) of a dielectric vertex in K'u = 2 f(delta) - f(2 delta),
// f(m delta) the mean of the normal field at x + m delta n and x - m delta n
__host__ __device__ __forceinline__ double kp_weight(int k) { return k < 2 ? 1.0 : -0.5; }

namespace {

// ---------------------------------------------------------------- the quadratic map
// Six-node triangle: corners 0, 1, 2, then the midpoints of the edges 01, 12, 20.
// y(xi, eta) = sum_a N_a(xi, eta) P_a with the quadratic Lagrange functions N_a.
struct P6 {
    double p[6][3];
};

__device__ __forceinline__ void p6_load(const P1Data& D, int64_t T, P6& P)
{
    for (int a = 0; a < 6; ++a) {
        const double* q = D.nodes + 3 * (int64_t)D.tri6[6 * T + a];
        P.p[a][0] = q[0]; P.p[a][1] = q[1]; P.p[a][2] = q[2];
    }
}

// point, tangents d/dxi, d/deta of the map at (xi, eta)
__device__ __forceinline__ void p6_eval(const P6& P, double xi, double eta, double* y, double* t1, double* t2)
{
    const double l0 = 1.0 - xi - eta, l1 = xi, l2 = eta;
    const double N[6] = {l0 * (2.0 * l0 - 1.0), l1 * (2.0 * l1 - 1.0), l2 * (2.0 * l2 - 1.0),
                         4.0 * l0 * l1, 4.0 * l1 * l2, 4.0 * l2 * l0};
    const double Dx[6] = {-(4.0 * l0 - 1.0), 4.0 * l1 - 1.0, 0.0, 4.0 * (l0 - l1), 4.0 * l2, -4.0 * l2};
    const double De[6] = {-(4.0 * l0 - 1.0), 0.0, 4.0 * l2 - 1.0, -4.0 * l1, 4.0 * l1, 4.0 * (l0 - l2)};
    for (int c = 0; c < 3; ++c) {
        double a = 0.0, b = 0.0, d = 0.0;
        for (int k = 0; k < 6; ++k) {
            a = fma(N[k], P.p[k][c], a);
            b = fma(Dx[k], P.p[k][c], b);
            d = fma(De[k], P.p[k][c], d);
        }
        y[c] = a; t1[c] = b; t2[c] = d;
    }
}

__device__ __forceinline__ double area_element(const double* t1, const double* t2)
{
    const double cx = t1[1] * t2[2] - t1[2] * t2[1];
    const double cy = t1[2] * t2[0] - t1[0] * t2[2];
    const double cz = t1[0] * t2[1] - t1[1] * t2[0];
    return sqrt(cx * cx + cy * cy + cz * cz);
}

// ---------------------------------------------------------------- set-up kernels
// Per triangle: the regular rule's points and weights w_q J_q (node64 / node32), the
// circumcircle of the corners (classification header, and the geometry record's
// circumcentre and eta R for the chunk spheres of the packed kernel), and per corner
// the integral of its basis function over the triangle (neutrality weights).
__global__ void k_p1_geom(P1Data D, double eta, double* __restrict__ geo, double4* __restrict__ node64,
                          float4* __restrict__ node32, double4* __restrict__ hdr64, float4* __restrict__ hdr32,
                          double* __restrict__ corner_int, int* __restrict__ status)
{
    const int64_t T = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (T >= D.N) return;
    P6 P;
    p6_load(D, T, P);
    const double* a = P.p[0];
    const double* b = P.p[1];
    const double* c = P.p[2];
    double ab[3], ac[3], n[3];
    for (int k = 0; k < 3; ++k) { ab[k] = b[k] - a[k]; ac[k] = c[k] - a[k]; }
    n[0] = ab[1] * ac[2] - ab[2] * ac[1];
    n[1] = ab[2] * ac[0] - ab[0] * ac[2];
    n[2] = ab[0] * ac[1] - ab[1] * ac[0];
    const double nn = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
    if (!(nn > 0.0)) {
        atomicExch(status, 1);
        return;
    }
    // circumcentre a + (|ac|^2 (n x ab) + |ab|^2 (ac x n)) / (2 |n|^2)
    const double aa = ac[0] * ac[0] + ac[1] * ac[1] + ac[2] * ac[2];
    const double bb = ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2];
    const double nxab[3] = {n[1] * ab[2] - n[2] * ab[1], n[2] * ab[0] - n[0] * ab[2], n[0] * ab[1] - n[1] * ab[0]};
    const double acxn[3] = {ac[1] * n[2] - ac[2] * n[1], ac[2] * n[0] - ac[0] * n[2], ac[0] * n[1] - ac[1] * n[0]};
    double cc[3];
    for (int k = 0; k < 3; ++k) cc[k] = a[k] + (aa * nxab[k] + bb * acxn[k]) / (2.0 * nn);
    const double R = sqrt((cc[0] - a[0]) * (cc[0] - a[0]) + (cc[1] - a[1]) * (cc[1] - a[1]) +
                          (cc[2] - a[2]) * (cc[2] - a[2]));
    double* G = geo + GEO_STRIDE * T;
    for (int k = 0; k < 3; ++k) {
        G[GEO_A + k] = a[k]; G[GEO_B + k] = b[k]; G[GEO_C + k] = c[k];
        G[GEO_N + k] = n[k] / sqrt(nn);
        G[GEO_CC + k] = cc[k];
        G[GEO_CTR + k] = (a[k] + b[k] + c[k]) / 3.0;
    }
    G[GEO_AREA] = 0.5 * sqrt(nn);
    G[GEO_R] = R;
    G[GEO_ETAR] = eta * R;
    const double e2 = (eta * R) * (eta * R);
    hdr64[T] = make_double4(cc[0], cc[1], cc[2], e2);
    hdr32[T] = make_float4(__double2float_rn(cc[0]), __double2float_rn(cc[1]), __double2float_rn(cc[2]),
                           __double2float_rn(e2));
    // regular rule: (xi, eta) = (s (1 - t), s t), weight ws wt s
    double ci[3] = {0.0, 0.0, 0.0};
    const int g = D.g;
    for (int i = 0; i < g; ++i)
        for (int j = 0; j < g; ++j) {
            const double s = D.rule[i], t = D.rule[j], w = D.rule[g + i] * D.rule[g + j] * s;
            const double xi = s * (1.0 - t), et = s * t;
            double y[3], t1[3], t2[3];
            p6_eval(P, xi, et, y, t1, t2);
            const double wj = w * area_element(t1, t2);
            const int q = i * g + j;
            node64[T * D.Q + q] = make_double4(y[0], y[1], y[2], wj);
            node32[T * D.Q + q] = make_float4(__double2float_rn(y[0]), __double2float_rn(y[1]),
                                              __double2float_rn(y[2]), __double2float_rn(wj));
            ci[0] += wj * (1.0 - xi - et);
            ci[1] += wj * xi;
            ci[2] += wj * et;
        }
    corner_int[3 * T] = ci[0];
    corner_int[3 * T + 1] = ci[1];
    corner_int[3 * T + 2] = ci[2];
}

// basis values of the regular rule's points (the same for every triangle)
__global__ void k_p1_lam(P1Data D)
{
    const int q = threadIdx.x;
    if (q >= D.Q) return;
    const int i = q / D.g, j = q % D.g;
    const double s = D.rule[i], t = D.rule[j];
    const double xi = s * (1.0 - t), et = s * t;
    D.lam[3 * q] = 1.0 - xi - et;
    D.lam[3 * q + 1] = xi;
    D.lam[3 * q + 2] = et;
}

// vertex targets of the products: (x, y, z, -) in FP64 and FP32
__global__ void k_p1_targets(P1Data D, double4* __restrict__ t64, float4* __restrict__ t32)
{
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= D.nv) return;
    const double* x = D.nodes + 3 * v;
    t64[v] = make_double4(x[0], x[1], x[2], 0.0);
    t32[v] = make_float4(__double2float_rn(x[0]), __double2float_rn(x[1]), __double2float_rn(x[2]), 0.f);
}

// One warp per vertex: count (phase 0) or list (phase 1) the triangles whose pair
// with it is singular (the vertex is a corner) or near in the FP32 or the FP64
// classification.  Triangles ascend.
__global__ void k_p1_near_rows(P1Data D, int phase, const float4* __restrict__ t32,
                               const double4* __restrict__ t64, const float4* __restrict__ hdr32,
                               const double4* __restrict__ hdr64, int32_t* __restrict__ count,
                               const int64_t* __restrict__ ptr, int32_t* __restrict__ col,
                               uint8_t* __restrict__ flag)
{
    const int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (v >= D.nv) return;
    const float4 x32 = t32[v];
    const double4 x64 = t64[v];
    int64_t pos = phase ? ptr[v] : 0;
    int cnt = 0;
    for (int64_t T0 = 0; T0 < D.N; T0 += 32) {
        const int64_t T = T0 + lane;
        uint8_t f = 0;
        if (T < D.N) {
            const int32_t* t6 = D.tri6 + 6 * T;
            const bool sing = t6[0] == v || t6[1] == v || t6[2] == v;
            const bool n32 = !is_far32(x32.x, x32.y, x32.z, hdr32[T]);
            const bool n64 = !is_far64(x64.x, x64.y, x64.z, hdr64[T]);
            f = (uint8_t)((n32 || sing ? 1 : 0) | (n64 || sing ? 2 : 0) | (sing ? 4 : 0));
        }
        const unsigned bal = __ballot_sync(0xffffffffu, f != 0);
        if (phase && f) {
            const int64_t k = pos + __popc(bal & ((1u << lane) - 1u));
            col[k] = (int32_t)T;
            flag[k] = f;
        }
        pos += __popc(bal);
        cnt += __popc(bal);
    }
    if (!phase && lane == 0) count[v] = cnt;
}

// ---------------------------------------------------------------- pair integrals
// Warp-wide FP64 integrals over one curved triangle T of the three basis functions,
// at a point x off the triangle or at one of its corners:
//   S[k] = int lambda_k / (4 pi |x - y|) dS_y,   G[k][c] = int lambda_k (x - y)_c / (4 pi |x - y|^3) dS_y.
// Every lane takes quadrature points; the sums are reduced over the warp (butterfly)
// and returned to every lane.

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Duffy rule on the reference sub-triangle (P0, P1, P2) collapsed at P0: points
// P0 + s (P1 - P0) + s t (P2 - P1), weight ws wt s |det(P1 - P0, P2 - P1)|.  The
// radial variable s runs over the pieces [e_k, e_{k+1}] of `edges` (nb pieces) with
// ns Gauss points each; t has nt points.  Adds to S, G (lane partials).
__device__ void duffy_part(const P6& P, const double* x, const double* P0, const double* P1,
                           const double* P2, const double* edges, int nb, const double* rs, int ns,
                           const double* rt, int nt, bool want_G, double* S, double (*G)[3])
{
    const double e1[2] = {P1[0] - P0[0], P1[1] - P0[1]};
    const double e2[2] = {P2[0] - P1[0], P2[1] - P1[1]};
    const double det = fabs(e1[0] * e2[1] - e1[1] * e2[0]);
    if (!(det > 0.0)) return;
    const int lane = threadIdx.x & 31;
    const int per = ns * nt;
    for (int k = lane; k < nb * per; k += 32) {
        const int piece = k / per, r = k - piece * per;
        const int i = r / nt, j = r - i * nt;
        const double lo = edges[piece], hi = edges[piece + 1];
        const double s = lo + (hi - lo) * rs[i];
        const double w = (hi - lo) * rs[ns + i] * rt[nt + j] * s * det;
        const double t = rt[j];
        const double xi = P0[0] + s * e1[0] + s * t * e2[0];
        const double et = P0[1] + s * e1[1] + s * t * e2[1];
        double y[3], t1[3], t2[3];
        p6_eval(P, xi, et, y, t1, t2);
        const double wj = w * area_element(t1, t2);
        const double d[3] = {x[0] - y[0], x[1] - y[1], x[2] - y[2]};
        const double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        const double ri = 1.0 / sqrt(r2);
        const double lamv[3] = {1.0 - xi - et, xi, et};
        const double a = wj * ri;
        for (int q = 0; q < 3; ++q) S[q] = fma(a, lamv[q], S[q]);
        if (want_G) {
            const double a3 = a * ri * ri;
            for (int q = 0; q < 3; ++q)
                for (int c = 0; c < 3; ++c) G[q][c] = fma(a3 * lamv[q], d[c], G[q][c]);
        }
    }
}

// reference point of the curved triangle nearest to x: the best of a grid sample
// (k = 12: the points (i/12, j/12), i + j <= 12), then projected Gauss-Newton steps
// on |y(xi, eta) - x|^2 (normal equations of the 3 x 2 least-squares step, the
// iterate projected back onto the reference triangle).  Every lane returns it.
__device__ void closest_ref(const P6& P, const double* x, double* out)
{
    const int lane = threadIdx.x & 31;
    const int K = 12;
    double best = 1e300;
    int bi = 1 << 30;
    for (int m = lane; m < (K + 1) * (K + 2) / 2; m += 32) {
        // m -> (i, j) in the order i = 0..K, j = 0..K-i
        int i = 0, rem = m;
        while (rem > K - i) { rem -= K - i + 1; ++i; }
        const int j = rem;
        double y[3], t1[3], t2[3];
        p6_eval(P, (double)i / K, (double)j / K, y, t1, t2);
        const double d2 = (y[0] - x[0]) * (y[0] - x[0]) + (y[1] - x[1]) * (y[1] - x[1]) + (y[2] - x[2]) * (y[2] - x[2]);
        if (d2 < best || (d2 == best && m < bi)) { best = d2; bi = m; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob < best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    int i = 0, rem = bi;
    while (rem > K - i) { rem -= K - i + 1; ++i; }
    double p[2] = {(double)i / K, (double)rem / K};
    for (int it = 0; it < 30; ++it) {
        double y[3], t1[3], t2[3];
        p6_eval(P, p[0], p[1], y, t1, t2);
        const double F[3] = {y[0] - x[0], y[1] - x[1], y[2] - x[2]};
        const double a11 = t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2];
        const double a12 = t1[0] * t2[0] + t1[1] * t2[1] + t1[2] * t2[2];
        const double a22 = t2[0] * t2[0] + t2[1] * t2[1] + t2[2] * t2[2];
        const double b1 = -(t1[0] * F[0] + t1[1] * F[1] + t1[2] * F[2]);
        const double b2 = -(t2[0] * F[0] + t2[1] * F[1] + t2[2] * F[2]);
        const double det = a11 * a22 - a12 * a12;
        if (!(det > 0.0)) break;
        double q0 = p[0] + (a22 * b1 - a12 * b2) / det;
        double q1 = p[1] + (a11 * b2 - a12 * b1) / det;
        // projection onto the reference triangle
        if (q0 + q1 > 1.0) {
            const double dd = 0.5 * (q0 + q1 - 1.0);
            q0 -= dd;
            q1 -= dd;
        }
        q0 = fmax(q0, 0.0);
        q1 = fmax(q1, 0.0);
        if (q0 + q1 > 1.0) {
            const double sum = q0 + q1;
            q0 /= sum;
            q1 /= sum;
        }
        const double step = sqrt((q0 - p[0]) * (q0 - p[0]) + (q1 - p[1]) * (q1 - p[1]));
        p[0] = q0;
        p[1] = q1;
        if (step < 1e-15) break;
    }
    out[0] = p[0];
    out[1] = p[1];
}

// The basis integrals of triangle T at x (warp-wide).  corner >= 0: x is that corner
// (singular rule); otherwise the near-singular rule.  Results on every lane.
__device__ void p1_pair(const P1Data& D, int64_t T, const double* x, int corner, bool want_G, double* S,
                        double (*G)[3])
{
    P6 P;
    p6_load(D, T, P);
    const double C[3][2] = {{0.0, 0.0}, {1.0, 0.0}, {0.0, 1.0}};
    double s[3] = {0.0, 0.0, 0.0}, g[3][3] = {{0.0}};
    if (corner >= 0) {
        const double edges[2] = {0.0, 1.0};
        duffy_part(P, x, C[corner], C[(corner + 1) % 3], C[(corner + 2) % 3], edges, 1, D.sing_rule, D.sing_n,
                   D.sing_rule, D.sing_n, want_G, s, g);
    } else {
        double p[2];
        closest_ref(P, x, p);
        double yp[3], t1[3], t2[3];
        p6_eval(P, p[0], p[1], yp, t1, t2);
        double size = 0.0;
        for (int a = 0; a < 3; ++a) {
            const double dd = sqrt((P.p[a][0] - yp[0]) * (P.p[a][0] - yp[0]) + (P.p[a][1] - yp[1]) * (P.p[a][1] - yp[1]) +
                                   (P.p[a][2] - yp[2]) * (P.p[a][2] - yp[2]));
            size = fmax(size, dd);
        }
        const double dist = sqrt((x[0] - yp[0]) * (x[0] - yp[0]) + (x[1] - yp[1]) * (x[1] - yp[1]) +
                                 (x[2] - yp[2]) * (x[2] - yp[2]));
        const double s_min = 0.1 * dist / size;
        // radial pieces: [0, q^m], [q^m, q^(m-1)], ..., [q, 1] with q = 0.2
        const double q = 0.2;
        int m = 0;
        if (!(s_min > 0.0)) m = 60;  // x on the surface: the deepest refinement
        else if (s_min < 1.0) m = min(60, (int)ceil(log(s_min) / log(q)));
        double edges[62];
        edges[0] = 0.0;
        for (int k = 0; k <= m; ++k) edges[k + 1] = pow(q, (double)(m - k));
        for (int k = 0; k < 3; ++k)
            duffy_part(P, x, p, C[k], C[(k + 1) % 3], edges, m + 1, D.near_rule, D.near_n, D.near_trule,
                       D.near_nt, want_G, s, g);
    }
    const double k4 = kInv4Pi;
    for (int k = 0; k < 3; ++k) {
        S[k] = k4 * warp_sum(s[k]);
        if (want_G)
            for (int c = 0; c < 3; ++c) G[k][c] = k4 * warp_sum(g[k][c]);
    }
}

// one warp per near pair of the vertices: its three basis integrals
__global__ void k_p1_near_values(P1Data D, const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                 const uint8_t* __restrict__ flag, double* __restrict__ val)
{
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= D.nnz) return;
    // the vertex of entry w: binary search in ptr
    int64_t lo = 0, hi = D.nv - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (ptr[mid] <= w) lo = mid; else hi = mid - 1;
    }
    const int64_t v = lo, T = col[w];
    const int32_t* t6 = D.tri6 + 6 * T;
    const int corner = (flag[w] & 4) ? (t6[0] == v ? 0 : (t6[1] == v ? 1 : 2)) : -1;
    const double x[3] = {D.nodes[3 * v], D.nodes[3 * v + 1], D.nodes[3 * v + 2]};
    double S[3], G[3][3];
    p1_pair(D, T, x, corner, false, S, G);
    if (lane == 0) {
        val[3 * w] = S[0];
        val[3 * w + 1] = S[1];
        val[3 * w + 2] = S[2];
    }
}

// Dielectric rows: one warp per point of the dielectric vertices (4 per vertex):
// count (phase 0) or list (phase 1) the triangles near it in the FP32 or the FP64
// classification.  Triangles ascend.
__global__ void k_p1_dnear_rows(P1Data D, int phase, const float4* __restrict__ hdr32,
                                const double4* __restrict__ hdr64, int32_t* __restrict__ count)
{
    const int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= 4 * D.nd) return;
    const double* x = D.dpts + 3 * p;
    const float xf = __double2float_rn(x[0]), yf = __double2float_rn(x[1]), zf = __double2float_rn(x[2]);
    int64_t pos = phase ? D.dptr[p] : 0;
    int cnt = 0;
    for (int64_t T0 = 0; T0 < D.N; T0 += 32) {
        const int64_t T = T0 + lane;
        uint8_t f = 0;
        if (T < D.N) {
            const bool n32 = !is_far32(xf, yf, zf, hdr32[T]);
            const bool n64 = !is_far64(x[0], x[1], x[2], hdr64[T]);
            f = (uint8_t)((n32 ? 1 : 0) | (n64 ? 2 : 0));
        }
        const unsigned bal = __ballot_sync(0xffffffffu, f != 0);
        if (phase && f) {
            const int64_t k = pos + __popc(bal & ((1u << lane) - 1u));
            D.dcol[k] = (int32_t)T;
            D.dflag[k] = f;
        }
        pos += __popc(bal);
        cnt += __popc(bal);
    }
    if (!phase && lane == 0) count[p] = cnt;
}

// one warp per near pair of a dielectric vertex's point: the weighted normal field of
// the three basis functions, kp_weight(k) G_j(x) . n_i
__global__ void k_p1_dnear_values(P1Data D)
{
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= D.dnnz) return;
    int64_t lo = 0, hi = 4 * D.nd - 1;  // the point of entry w
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (D.dptr[mid] <= w) lo = mid; else hi = mid - 1;
    }
    const int64_t p = lo, d = p >> 2;
    const double x[3] = {D.dpts[3 * p], D.dpts[3 * p + 1], D.dpts[3 * p + 2]};
    const double* n = D.dnrm + 3 * d;
    double S[3], G[3][3];
    p1_pair(D, D.dcol[w], x, -1, true, S, G);
    if (lane == 0) {
        const double c = kp_weight((int)(p & 3));
        for (int k = 0; k < 3; ++k) D.dval[3 * w + k] = c * (G[k][0] * n[0] + G[k][1] * n[1] + G[k][2] * n[2]);
    }
}

}  // namespace

namespace {

// ---------------------------------------------------------------- products
// The density folded into the regular rule's weights: w_q J_q sum_k lambda_k(q) x_{v_k}
// (FP32 stream for the packed kernel, FP64 stream for the FP64 kernel).
__global__ void k_p1_fold(P1Data D, const double4* __restrict__ node64, const double* __restrict__ x,
                          float4* __restrict__ q32, double4* __restrict__ q64)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= D.N * D.Q) return;
    const int64_t T = i / D.Q;
    const int q = (int)(i - T * D.Q);
    const int32_t* t6 = D.tri6 + 6 * T;
    const double dens = D.lam[3 * q] * x[t6[0]] + D.lam[3 * q + 1] * x[t6[1]] + D.lam[3 * q + 2] * x[t6[2]];
    const double4 nd = node64[i];
    const double w = nd.w * dens;
    if (q32) q32[i] = make_float4(__double2float_rn(nd.x), __double2float_rn(nd.y), __double2float_rn(nd.z),
                                  __double2float_rn(w));
    if (q64) q64[i] = make_double4(nd.x, nd.y, nd.z, w);
}

// One warp per collocation point (vertex) v: the regular pairs' potential from the
// slices' partial sums, the singular and near-singular pairs from the CSR (those the
// product's own classification left out: bit 0 for FP32, bit 1 for FP64), then the
// row equation.  The row has a single owner, so nothing collides.
__global__ void k_p1_rows(P1Data D, int splits, const double* __restrict__ part, uint8_t bit,
                          const double* __restrict__ x, int64_t nunk, double* __restrict__ y)
{
    const int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (v >= D.nv || D.vkind[v] == BEM_DIELECTRIC) return;  // dielectric rows: k_p1_diel_rows
    double f = 0.0;
    for (int s = lane; s < splits; s += 32) f += part[((int64_t)s * D.nv + v) * 4];
    f *= kInv4Pi;
    for (int64_t e = D.ptr[v] + lane; e < D.ptr[v + 1]; e += 32) {
        if (!(D.flag[e] & bit)) continue;
        const int32_t* t6 = D.tri6 + 6 * (int64_t)D.col[e];
        const double* vv = D.val + 3 * e;
        f = fma(vv[0], x[t6[0]], fma(vv[1], x[t6[1]], fma(vv[2], x[t6[2]], f)));
    }
    f = warp_sum(f);
    if (lane == 0) {
        if (D.vkind[v] == BEM_FLOATING) f -= x[D.nv + D.vaux[v]];
        y[v] = f;
    }
}

// Dielectric rows (Eq. Final3), one warp per dielectric vertex i:
//   y_i = (eps+ + eps-)/2 x_i + (eps+ - eps-) (K'x)_i,
//   (K'x)_i = sum_k kp_weight(k) E(p_k) . n_i over its four points p_k,
// E from the regular pairs' partial sums of the points (field components 1..3) and
// the near pairs' CSR values (those the product's classification left out).
__global__ void k_p1_diel_rows(P1Data D, int splits, const double* __restrict__ part, uint8_t bit,
                               const double* __restrict__ x, double* __restrict__ y)
{
    const int64_t d = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (d >= D.nd) return;
    const int64_t M4 = 4 * D.nd;
    const double* n = D.dnrm + 3 * d;
    double f = 0.0;
    for (int i = lane; i < 4 * splits; i += 32) {
        const int k = i & 3, sp = i >> 2;
        const double* q = part + ((int64_t)sp * M4 + 4 * d + k) * 4;
        f = fma(kp_weight(k), q[1] * n[0] + q[2] * n[1] + q[3] * n[2], f);
    }
    f *= kInv4Pi;
    for (int k = 0; k < 4; ++k) {
        const int64_t p = 4 * d + k;
        for (int64_t e = D.dptr[p] + lane; e < D.dptr[p + 1]; e += 32) {
            if (!(D.dflag[e] & bit)) continue;
            const int32_t* t6 = D.tri6 + 6 * (int64_t)D.dcol[e];
            const double* vv = D.dval + 3 * e;
            f = fma(vv[0], x[t6[0]], fma(vv[1], x[t6[1]], fma(vv[2], x[t6[2]], f)));
        }
    }
    f = warp_sum(f);
    if (lane == 0) {
        const int64_t v = D.dvert[d];
        y[v] = fma(D.dcoef[2 * v], x[v], D.dcoef[2 * v + 1] * f);
    }
}

// neutrality rows (Eq. Final4 by Gauss's law): y_{nv+f} = sum_v a_f[v] x_v, one block
// per floating body, fixed summation order
__global__ void k_p1_neutral(P1Data D, const double* __restrict__ x, double* __restrict__ y)
{
    __shared__ double sh[256];
    const int f = blockIdx.x;
    const double* a = D.neut_w + (int64_t)f * D.nv;
    double s = 0.0;
    for (int64_t v = threadIdx.x; v < D.nv; v += 256) s = fma(a[v], x[v], s);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) y[D.nv + f] = sh[0];
}

// b: V0 on conductor rows, 0 elsewhere
__global__ void k_p1_rhs(P1Data D, int64_t nunk, int nreg, const double* __restrict__ V0, double* __restrict__ b)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nunk) return;
    b[i] = (i < D.nv && D.vkind[i] == BEM_CONDUCTOR) ? V0[D.vaux[i]] : 0.0;
}

// Jacobi scaling: 1 / v_vv (the singular pairs' own-corner integrals), 1 on the
// neutrality rows
__global__ void k_p1_jacobi(P1Data D, int64_t nunk, double* __restrict__ jinv)
{
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= nunk) return;
    if (v >= D.nv) {
        jinv[v] = 1.0;
        return;
    }
    if (D.vkind[v] == BEM_DIELECTRIC) {  // the jump term (eps+ + eps-)/2
        jinv[v] = 1.0 / D.dcoef[2 * v];
        return;
    }
    double d = 0.0;
    for (int64_t e = D.ptr[v]; e < D.ptr[v + 1]; ++e) {
        if (!(D.flag[e] & 4)) continue;
        const int32_t* t6 = D.tri6 + 6 * (int64_t)D.col[e];
        for (int k = 0; k < 3; ++k)
            if (t6[k] == v) d += D.val[3 * e + k];
    }
    jinv[v] = d != 0.0 ? 1.0 / d : 1.0;
}

// Dense rows [row0, row1) of the collocation matrix: one thread per collocation point
// loops over all triangles and adds each regular pair's three basis integrals to its
// own row (the paper's collision-free ownership), then the CSR's pairs and the row
// equation; neutrality rows from their weights.  F32: regular pairs in FP32.
template <bool F32>
__global__ void k_p1_assemble(P1Data D, int64_t row0, int64_t row1, const double4* __restrict__ node64,
                              const double4* __restrict__ hdr64, const float4* __restrict__ hdr32,
                              double* __restrict__ A, int64_t lda, int64_t nunk)
{
    const int64_t r = row0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= row1) return;
    double* row = A + (r - row0) * lda;
    for (int64_t j = 0; j < nunk; ++j) row[j] = 0.0;
    if (r >= D.nv) {
        const double* a = D.neut_w + (r - D.nv) * D.nv;
        for (int64_t v = 0; v < D.nv; ++v) row[v] = a[v];
        return;
    }
    const uint8_t bit = F32 ? 1 : 2;
    if (D.vkind[r] == BEM_DIELECTRIC) {
        // (eps+ + eps-)/2 e_r + (eps+ - eps-) K'_r: the normal field of every basis
        // function at the vertex's four points, weighted
        const int64_t d = D.didx[r];
        const double* n = D.dnrm + 3 * d;
        const double B = D.dcoef[2 * r + 1];
        for (int k = 0; k < 4; ++k) {
            const double* p = D.dpts + 3 * (4 * d + k);
            const float pf[3] = {__double2float_rn(p[0]), __double2float_rn(p[1]), __double2float_rn(p[2])};
            const double c = kp_weight(k) * B * kInv4Pi;
            for (int64_t T = 0; T < D.N; ++T) {
                const bool far = F32 ? is_far32(pf[0], pf[1], pf[2], hdr32[T]) : is_far64(p[0], p[1], p[2], hdr64[T]);
                if (!far) continue;
                double s[3] = {0.0, 0.0, 0.0};
                for (int q = 0; q < D.Q; ++q) {
                    const double4 nd = node64[T * D.Q + q];
                    double a;
                    if (F32) {
                        const float dx = pf[0] - __double2float_rn(nd.x), dy = pf[1] - __double2float_rn(nd.y),
                                    dz = pf[2] - __double2float_rn(nd.z);
                        const float ri = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                        const float dn = fmaf(dx, (float)n[0], fmaf(dy, (float)n[1], dz * (float)n[2]));
                        a = (double)(__double2float_rn(nd.w) * ri * ri * ri * dn);
                    } else {
                        const double dx = p[0] - nd.x, dy = p[1] - nd.y, dz = p[2] - nd.z;
                        const double r2 = dx * dx + dy * dy + dz * dz;
                        a = nd.w * (dx * n[0] + dy * n[1] + dz * n[2]) / (r2 * sqrt(r2));
                    }
                    for (int kk = 0; kk < 3; ++kk) s[kk] = fma(a, D.lam[3 * q + kk], s[kk]);
                }
                const int32_t* t6 = D.tri6 + 6 * T;
                for (int kk = 0; kk < 3; ++kk) row[t6[kk]] += c * s[kk];
            }
            for (int64_t e = D.dptr[4 * d + k]; e < D.dptr[4 * d + k + 1]; ++e) {
                if (!(D.dflag[e] & bit)) continue;
                const int32_t* t6 = D.tri6 + 6 * (int64_t)D.dcol[e];
                for (int kk = 0; kk < 3; ++kk) row[t6[kk]] += B * D.dval[3 * e + kk];
            }
        }
        row[r] += D.dcoef[2 * r];
        return;
    }
    const double* xv = D.nodes + 3 * r;
    const float xf = __double2float_rn(xv[0]), yf = __double2float_rn(xv[1]), zf = __double2float_rn(xv[2]);
    for (int64_t T = 0; T < D.N; ++T) {
        const bool far = F32 ? is_far32(xf, yf, zf, hdr32[T]) : is_far64(xv[0], xv[1], xv[2], hdr64[T]);
        if (!far) continue;
        double s[3] = {0.0, 0.0, 0.0};
        for (int q = 0; q < D.Q; ++q) {
            const double4 nd = node64[T * D.Q + q];
            double a;
            if (F32) {
                const float dx = xf - __double2float_rn(nd.x), dy = yf - __double2float_rn(nd.y),
                            dz = zf - __double2float_rn(nd.z);
                a = (double)(__double2float_rn(nd.w) * rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz))));
            } else {
                const double dx = xv[0] - nd.x, dy = xv[1] - nd.y, dz = xv[2] - nd.z;
                a = nd.w / sqrt(dx * dx + dy * dy + dz * dz);
            }
            for (int k = 0; k < 3; ++k) s[k] = fma(a, D.lam[3 * q + k], s[k]);
        }
        const int32_t* t6 = D.tri6 + 6 * T;
        for (int k = 0; k < 3; ++k) row[t6[k]] += kInv4Pi * s[k];
    }
    for (int64_t e = D.ptr[r]; e < D.ptr[r + 1]; ++e) {
        if (!(D.flag[e] & bit)) continue;
        const int32_t* t6 = D.tri6 + 6 * (int64_t)D.col[e];
        for (int k = 0; k < 3; ++k) row[t6[k]] += D.val[3 * e + k];
    }
    if (D.vkind[r] == BEM_FLOATING) row[D.nv + D.vaux[r]] = -1.0;
}

// The deferred near pass of the field at arbitrary points: one warp per point finds
// the triangles the product's classification left out (FP32 or FP64) and adds their
// near-singular integrals of phi and E with the density u, to the slices' sums.
template <bool F32>
__global__ void k_p1_points_near(P1Data D, int64_t M, int splits, const double* __restrict__ pts,
                                 const float4* __restrict__ hdr32, const double4* __restrict__ hdr64,
                                 const double* __restrict__ u, const double* __restrict__ part,
                                 double* __restrict__ phi, double* __restrict__ E)
{
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= M) return;
    const double x[3] = {pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]};
    const float xf = __double2float_rn(x[0]), yf = __double2float_rn(x[1]), zf = __double2float_rn(x[2]);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int s = lane; s < splits; s += 32)
        for (int c = 0; c < 4; ++c) acc[c] += part[((int64_t)s * M + i) * 4 + c];
    for (int c = 0; c < 4; ++c) acc[c] = kInv4Pi * warp_sum(acc[c]);
    for (int64_t T0 = 0; T0 < D.N; T0 += 32) {
        const int64_t T = T0 + lane;
        bool nr = false;
        if (T < D.N) nr = F32 ? !is_far32(xf, yf, zf, hdr32[T]) : !is_far64(x[0], x[1], x[2], hdr64[T]);
        unsigned bal = __ballot_sync(0xffffffffu, nr);
        while (bal) {
            const int b = __ffs(bal) - 1;
            bal &= bal - 1;
            const int64_t Tn = T0 + b;
            double S[3], G[3][3];
            p1_pair(D, Tn, x, -1, true, S, G);
            const int32_t* t6 = D.tri6 + 6 * Tn;
            for (int k = 0; k < 3; ++k) {
                const double uk = u[t6[k]];
                acc[0] = fma(uk, S[k], acc[0]);
                for (int c = 0; c < 3; ++c) acc[1 + c] = fma(uk, G[k][c], acc[1 + c]);
            }
        }
    }
    if (lane == 0) {
        if (phi) phi[i] = acc[0];
        if (E) {
            E[3 * i] = acc[1];
            E[3 * i + 1] = acc[2];
            E[3 * i + 2] = acc[3];
        }
    }
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// ---------------------------------------------------------------- host side
template <class T>
static int p1_alloc(bem_ctx* c, T** p, size_t n)
{
    if (cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_err(c, BEM_ERR_NOMEM, "P1 set-up: cudaMalloc of %zu bytes failed", n * sizeof(T));
    }
    return BEM_OK;
}

void p1_free(bem_ctx* c)
{
    P1Data* D = c->p1;
    if (!D) return;
    void* ptrs[] = {D->nodes, D->tri6, D->lam, D->rule, D->sing_rule, D->near_rule, D->near_trule, D->ptr,
                    D->col, D->flag, D->val, D->neut_w, D->vkind, D->vaux, D->phi_all, D->ones, D->d_region,
                    D->dvert, D->didx, D->dpts, D->dnrm, D->dcoef, D->dptr, D->dcol, D->dflag, D->dval};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->qnode64) cudaFree(c->qnode64);
    c->qnode64 = nullptr;
    delete D;
    c->p1 = nullptr;
}

// Gauss-Legendre on [0, 1]: points then weights
static std::vector<double> gl01(int n)
{
    std::vector<double> x, w;
    gauss_legendre_pm1(n, x, w);
    std::vector<double> out(2 * n);
    for (int i = 0; i < n; ++i) {
        out[i] = 0.5 * (x[i] + 1.0);
        out[n + i] = 0.5 * w[i];
    }
    return out;
}

int p1_matvec_impl(bem_ctx* c, int precision, int nrhs, const double* x, double* y)
{
    if (precision != BEM_FP64 && precision != BEM_MIXED)
        return set_err(c, BEM_ERR_ARG, "P1 products: precision must be BEM_FP64 or BEM_MIXED");
    P1Data& D = *c->p1;
    cudaStream_t s = c->stream;
    const int64_t nv = D.nv, n = c->nunk;
    const int splits = far_splits(c, precision, nv);
    if ((size_t)splits * nv * 4 > c->part_cap) return set_err(c, BEM_ERR_CAPACITY, "far workspace too small");
    for (int r = 0; r < nrhs; ++r) {
        const double* xr = x + (int64_t)r * n;
        double* yr = y + (int64_t)r * n;
        const bool f32 = precision == BEM_MIXED;
        k_p1_fold<<<nblk(D.N * D.Q, 256), 256, 0, s>>>(D, c->node64, xr, f32 ? c->qnode : nullptr,
                                                       f32 ? nullptr : c->qnode64);
        BEM_LAUNCH_CHECK(c);
        // every row needs phi alone: the packed kernel's phi-only tiles
        FarTargets T{c->tgt32, nullptr, c->tgt64, nullptr, nv, D.phi_all};
        int rc = launch_far(c, precision, T, c->ones, 1, 0, splits, c->part);
        if (rc) return rc;
        c->cnt.matvecs[precision] += 1;
        k_p1_rows<<<nblk(nv * 32, 128), 128, 0, s>>>(D, splits, c->part, (uint8_t)(f32 ? 1 : 2), xr, n, yr);
        BEM_LAUNCH_CHECK(c);
        if (D.nd > 0) {
            // the dielectric vertices' four points: regular pairs' field by the far kernel
            // (the partial sums of the vertex targets have been read), then the rows
            const int64_t M4 = 4 * D.nd;
            const int sp4 = far_splits(c, precision, M4);
            FarTargets T4{nullptr, nullptr, nullptr, D.dpts, M4};
            if ((rc = launch_far(c, precision, T4, c->ones, 1, 0, sp4, c->part))) return rc;
            k_p1_diel_rows<<<nblk(D.nd * 32, 128), 128, 0, s>>>(D, sp4, c->part, (uint8_t)(f32 ? 1 : 2), xr, yr);
            BEM_LAUNCH_CHECK(c);
        }
        if (c->nfloat > 0) {
            k_p1_neutral<<<c->nfloat, 256, 0, s>>>(D, xr, yr);
            BEM_LAUNCH_CHECK(c);
        }
    }
    return BEM_OK;
}

int p1_rhs(bem_ctx* c, int nrhs, const double* V0, double* b)
{
    P1Data& D = *c->p1;
    const int nreg = (int)c->regions.size();
    const double* v = V0 ? V0 : c->region_V0;
    for (int r = 0; r < nrhs; ++r) {
        k_p1_rhs<<<nblk(c->nunk, 256), 256, 0, c->stream>>>(D, c->nunk, nreg, v + (int64_t)r * nreg,
                                                           b + (int64_t)r * c->nunk);
        BEM_LAUNCH_CHECK(c);
    }
    return BEM_OK;
}

int p1_eval_field(bem_ctx* c, int precision, const double* u, int64_t M, const double* pts, double* phi,
                  double* E)
{
    P1Data& D = *c->p1;
    cudaStream_t s = c->stream;
    const bool f32 = precision == BEM_MIXED;
    k_p1_fold<<<nblk(D.N * D.Q, 256), 256, 0, s>>>(D, c->node64, u, f32 ? c->qnode : nullptr,
                                                   f32 ? nullptr : c->qnode64);
    BEM_LAUNCH_CHECK(c);
    const int64_t CH = c->prm.max_points;
    for (int64_t m0 = 0; m0 < M; m0 += CH) {
        const int64_t mc = std::min(CH, M - m0);
        const int splits = far_splits(c, precision, mc);
        if ((size_t)splits * mc * 4 > c->part_cap) return set_err(c, BEM_ERR_CAPACITY, "far workspace too small");
        FarTargets T{nullptr, nullptr, nullptr, pts + 3 * m0, mc};
        int rc = launch_far(c, precision, T, c->ones, 1, 0, splits, c->part);
        if (rc) return rc;
        if (f32)
            k_p1_points_near<true><<<nblk(mc * 32, 128), 128, 0, s>>>(D, mc, splits, pts + 3 * m0, c->hdr32, c->hdr64,
                                                                     u, c->part, phi ? phi + m0 : nullptr,
                                                                     E ? E + 3 * m0 : nullptr);
        else
            k_p1_points_near<false><<<nblk(mc * 32, 128), 128, 0, s>>>(D, mc, splits, pts + 3 * m0, c->hdr32,
                                                                      c->hdr64, u, c->part, phi ? phi + m0 : nullptr,
                                                                      E ? E + 3 * m0 : nullptr);
        BEM_LAUNCH_CHECK(c);
    }
    return BEM_OK;
}

int p1_assemble(bem_ctx* c, int64_t row0, int64_t row1, int precision, double* A, int64_t lda)
{
    P1Data& D = *c->p1;
    if (row1 <= row0) return BEM_OK;
    if (precision == BEM_MIXED)
        k_p1_assemble<true><<<nblk(row1 - row0, 64), 64, 0, c->stream>>>(D, row0, row1, c->node64, c->hdr64,
                                                                          c->hdr32, A, lda, c->nunk);
    else
        k_p1_assemble<false><<<nblk(row1 - row0, 64), 64, 0, c->stream>>>(D, row0, row1, c->node64, c->hdr64,
                                                                           c->hdr32, A, lda, c->nunk);
    BEM_LAUNCH_CHECK(c);
    return BEM_OK;
}

extern "C" void bem_p1_default_params(bem_p1_params* p)
{
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->eta = 4.0;
    p->far_order = 4;
    p->sing_order = 24;
    p->near_radial = 16;
    p->near_angular = 64;
    p->gmres_restart = 100;
    p->max_iters = 2000;
    p->max_refine = 6;
    p->max_points = 131072;
    p->far32_variant = 2;
}

// Unit normal of the six-node map of triangle t6 at its corner k: dy/dxi x dy/deta of
// the quadratic Lagrange map there, normalised.
static void corner_normal(const double* nodes, const int32_t* t6, int k, double* n)
{
    const double xi = k == 1 ? 1.0 : 0.0, eta = k == 2 ? 1.0 : 0.0;
    const double l0 = 1.0 - xi - eta, l1 = xi, l2 = eta;
    const double Dx[6] = {-(4.0 * l0 - 1.0), 4.0 * l1 - 1.0, 0.0, 4.0 * (l0 - l1), 4.0 * l2, -4.0 * l2};
    const double De[6] = {-(4.0 * l0 - 1.0), 0.0, 4.0 * l2 - 1.0, -4.0 * l1, 4.0 * l1, 4.0 * (l0 - l2)};
    double a[3] = {0.0, 0.0, 0.0}, b[3] = {0.0, 0.0, 0.0};
    for (int m = 0; m < 6; ++m)
        for (int c = 0; c < 3; ++c) {
            a[c] += Dx[m] * nodes[3 * (int64_t)t6[m] + c];
            b[c] += De[m] * nodes[3 * (int64_t)t6[m] + c];
        }
    n[0] = a[1] * b[2] - a[2] * b[1];
    n[1] = a[2] * b[0] - a[0] * b[2];
    n[2] = a[0] * b[1] - a[1] * b[0];
    const double l = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    for (int c = 0; c < 3; ++c) n[c] /= l;
}

// Dielectric rows: every dielectric vertex's normal (the sum of the unit normals its
// triangles have at that corner, normalised), its step delta = kDeltaRel times the
// mean length of the corner-to-corner edges at it, and its four points
// x +- delta n, x +- 2 delta n; then the near pairs of those points and their FP64
// near-singular normal fields.
constexpr double kDeltaRel = 1e-3;

static int p1_dielectric_setup(bem_ctx* c, const double* nodes, const int32_t* tri6,
                               const std::vector<int32_t>& vkind, const std::vector<int32_t>& vreg)
{
    P1Data& D = *c->p1;
    cudaStream_t s = c->stream;
    const int64_t nv = D.nv, N = D.N;
    std::vector<int32_t> dvert, didx(nv, -1);
    for (int64_t v = 0; v < nv; ++v)
        if (vkind[v] == BEM_DIELECTRIC) {
            didx[v] = (int32_t)dvert.size();
            dvert.push_back((int32_t)v);
        }
    D.nd = (int64_t)dvert.size();
    std::vector<double> coef(2 * nv, 0.0);
    for (int64_t v = 0; v < nv; ++v)
        if (vkind[v] == BEM_DIELECTRIC) {
            const bem_region& R = c->regions[vreg[v]];
            coef[2 * v] = 0.5 * (R.eps_plus + R.eps_minus);
            coef[2 * v + 1] = R.eps_plus - R.eps_minus;
        }
    int rc;
    if ((rc = p1_alloc(c, &D.didx, nv)) || (rc = p1_alloc(c, &D.dcoef, 2 * nv))) return rc;
    BEM_CUDA_TRY(c, cudaMemcpyAsync(D.didx, didx.data(), nv * 4, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(D.dcoef, coef.data(), 2 * nv * 8, cudaMemcpyHostToDevice, s));
    if (D.nd == 0) return cudaStreamSynchronize(s) == cudaSuccess ? BEM_OK : set_err(c, BEM_ERR_CUDA, "sync");
    // normals (triangles in order) and mean edge lengths (edges 01 of all triangles,
    // then 12, then 20)
    std::vector<double> nrm(3 * nv, 0.0), hsum(nv, 0.0), hcnt(nv, 0.0);
    for (int64_t T = 0; T < N; ++T)
        for (int k = 0; k < 3; ++k) {
            double n[3];
            corner_normal(nodes, tri6 + 6 * T, k, n);
            for (int cc = 0; cc < 3; ++cc) nrm[3 * (int64_t)tri6[6 * T + k] + cc] += n[cc];
        }
    for (int e = 0; e < 3; ++e)
        for (int64_t T = 0; T < N; ++T) {
            const int32_t a = tri6[6 * T + e], b = tri6[6 * T + (e + 1) % 3];
            double L = 0.0;
            for (int cc = 0; cc < 3; ++cc) L += (nodes[3 * a + cc] - nodes[3 * b + cc]) * (nodes[3 * a + cc] - nodes[3 * b + cc]);
            L = std::sqrt(L);
            hsum[a] += L; hsum[b] += L;
            hcnt[a] += 1.0; hcnt[b] += 1.0;
        }
    std::vector<double> dn(3 * D.nd), dp(12 * D.nd);
    for (int64_t d = 0; d < D.nd; ++d) {
        const int64_t v = dvert[d];
        const double* nv3 = &nrm[3 * v];
        const double l = std::sqrt(nv3[0] * nv3[0] + nv3[1] * nv3[1] + nv3[2] * nv3[2]);
        const double delta = kDeltaRel * hsum[v] / hcnt[v];
        for (int cc = 0; cc < 3; ++cc) dn[3 * d + cc] = nv3[cc] / l;
        const double m[4] = {1.0, -1.0, 2.0, -2.0};
        for (int k = 0; k < 4; ++k)
            for (int cc = 0; cc < 3; ++cc)
                dp[3 * (4 * d + k) + cc] = nodes[3 * v + cc] + m[k] * delta * dn[3 * d + cc];
    }
    const int64_t M4 = 4 * D.nd;
    int32_t* d_count = nullptr;
    if ((rc = p1_alloc(c, &D.dvert, D.nd)) || (rc = p1_alloc(c, &D.dnrm, 3 * D.nd)) ||
        (rc = p1_alloc(c, &D.dpts, 3 * M4)) || (rc = p1_alloc(c, &D.dptr, M4 + 1)) ||
        (rc = p1_alloc(c, &d_count, M4)))
        return rc;
    BEM_CUDA_TRY(c, cudaMemcpyAsync(D.dvert, dvert.data(), D.nd * 4, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(D.dnrm, dn.data(), 3 * D.nd * 8, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(D.dpts, dp.data(), 3 * M4 * 8, cudaMemcpyHostToDevice, s));
    k_p1_dnear_rows<<<nblk(M4 * 32, 128), 128, 0, s>>>(D, 0, c->hdr32, c->hdr64, d_count);
    cudaError_t e = cudaGetLastError();
    std::vector<int32_t> cnt(M4);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cnt.data(), d_count, M4 * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_count);
    if (e != cudaSuccess) return set_err(c, BEM_ERR_CUDA, "P1 dielectric near pairs: %s", cudaGetErrorString(e));
    std::vector<int64_t> ptr(M4 + 1, 0);
    for (int64_t p = 0; p < M4; ++p) ptr[p + 1] = ptr[p] + cnt[p];
    D.dnnz = ptr[M4];
    if ((rc = p1_alloc(c, &D.dcol, D.dnnz)) || (rc = p1_alloc(c, &D.dflag, D.dnnz)) ||
        (rc = p1_alloc(c, &D.dval, 3 * D.dnnz)))
        return rc;
    BEM_CUDA_TRY(c, cudaMemcpyAsync(D.dptr, ptr.data(), (M4 + 1) * 8, cudaMemcpyHostToDevice, s));
    k_p1_dnear_rows<<<nblk(M4 * 32, 128), 128, 0, s>>>(D, 1, c->hdr32, c->hdr64, nullptr);
    BEM_LAUNCH_CHECK(c);
    if (D.dnnz > 0) {
        k_p1_dnear_values<<<nblk(D.dnnz * 32, 128), 128, 0, s>>>(D);
        BEM_LAUNCH_CHECK(c);
    }
    BEM_CUDA_TRY(c, cudaStreamSynchronize(s));
    return BEM_OK;
}

static int p1_create_impl(bem_ctx* c, int64_t nn, const double* nodes, int64_t nv, int64_t N,
                          const int32_t* tri6, const int32_t* region, const bem_p1_params& p)
{
    cudaStream_t s = c->stream;
    P1Data* Dp = new P1Data();
    c->p1 = Dp;
    P1Data& D = *Dp;
    D.nn = nn;
    D.nv = nv;
    D.N = N;
    D.g = p.far_order;
    D.Q = p.far_order * p.far_order;
    D.sing_n = p.sing_order;
    D.near_n = p.near_radial;
    D.near_nt = p.near_angular;
    c->np = N;
    c->nv = nv;
    c->g = D.g;
    c->Q = D.Q;
    c->far32_tp = p.far32_variant;
    c->far_slots = 4;
    int rc;
    // rows: the region of every vertex (all its triangles must agree)
    std::vector<int32_t> vreg(nv, -1);
    for (int64_t T = 0; T < N; ++T)
        for (int k = 0; k < 3; ++k) {
            const int32_t v = tri6[6 * T + k];
            if (vreg[v] >= 0 && vreg[v] != region[T])
                return set_err(c, BEM_ERR_ARG, "P1: vertex %d lies on two regions", v);
            vreg[v] = region[T];
        }
    std::vector<int32_t> vkind(nv), vaux(nv), phi_all(nv, BEM_CONDUCTOR);
    for (int64_t v = 0; v < nv; ++v) {
        if (vreg[v] < 0) return set_err(c, BEM_ERR_ARG, "P1: vertex %lld is no triangle's corner", (long long)v);
        const bem_region& R = c->regions[vreg[v]];
        vkind[v] = R.kind;
        vaux[v] = R.kind == BEM_FLOATING ? R.floating_id : vreg[v];
    }
    // device copies and rules
    std::vector<double> r_reg = gl01(D.g), r_sing = gl01(D.sing_n), r_near = gl01(D.near_n), r_t = gl01(D.near_nt);
    if ((rc = p1_alloc(c, &D.nodes, 3 * nn)) || (rc = p1_alloc(c, &D.tri6, 6 * N)) ||
        (rc = p1_alloc(c, &D.lam, 3 * D.Q)) || (rc = p1_alloc(c, &D.rule, r_reg.size())) ||
        (rc = p1_alloc(c, &D.sing_rule, r_sing.size())) || (rc = p1_alloc(c, &D.near_rule, r_near.size())) ||
        (rc = p1_alloc(c, &D.near_trule, r_t.size())) || (rc = p1_alloc(c, &D.vkind, nv)) ||
        (rc = p1_alloc(c, &D.vaux, nv)) || (rc = p1_alloc(c, &D.phi_all, nv)) || (rc = p1_alloc(c, &D.ones, N)) ||
        (rc = p1_alloc(c, &D.d_region, N)) || (rc = p1_alloc(c, &c->geo, (size_t)GEO_STRIDE * N)) ||
        (rc = p1_alloc(c, &c->node64, (size_t)N * D.Q)) || (rc = p1_alloc(c, &c->node32, (size_t)N * D.Q)) ||
        (rc = p1_alloc(c, &c->qnode, (size_t)N * D.Q)) || (rc = p1_alloc(c, &c->qnode64, (size_t)N * D.Q)) ||
        (rc = p1_alloc(c, &c->hdr64, N)) || (rc = p1_alloc(c, &c->hdr32, N)) ||
        (rc = p1_alloc(c, &c->chunk_sph, (N + 31) / 32)) || (rc = p1_alloc(c, &c->tgt64, nv)) ||
        (rc = p1_alloc(c, &c->tgt32, nv)) || (rc = p1_alloc(c, &c->d_status, 1)) ||
        (rc = p1_alloc(c, &c->d_near_count, 4)))
        return rc;
    BEM_CUDA_TRY(c, cudaMemcpyAsync(D.nodes, nodes, 3 * nn * sizeof(double), cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(D.tri6, tri6, 6 * N * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(D.rule, r_reg.data(), r_reg.size() * 8, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(D.sing_rule, r_sing.data(), r_sing.size() * 8, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(D.near_rule, r_near.data(), r_near.size() * 8, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(D.near_trule, r_t.data(), r_t.size() * 8, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(D.vkind, vkind.data(), nv * 4, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(D.vaux, vaux.data(), nv * 4, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(D.phi_all, phi_all.data(), nv * 4, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(D.d_region, region, N * 4, cudaMemcpyHostToDevice, s));
    {
        std::vector<double> ones(N, 1.0);
        BEM_CUDA_TRY(c, cudaMemcpyAsync(D.ones, ones.data(), N * 8, cudaMemcpyHostToDevice, s));
        BEM_CUDA_TRY(c, cudaStreamSynchronize(s));
    }
    c->ones = D.ones;
    BEM_CUDA_TRY(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), s));
    BEM_CUDA_TRY(c, cudaMemsetAsync(c->d_near_count, 0, 4 * sizeof(unsigned long long), s));
    k_p1_lam<<<1, 64, 0, s>>>(D);
    BEM_LAUNCH_CHECK(c);
    std::vector<double> cint(3 * N);
    {
        double* d_cint = nullptr;
        if ((rc = p1_alloc(c, &d_cint, 3 * N))) return rc;
        k_p1_geom<<<nblk(N, 128), 128, 0, s>>>(D, p.eta, c->geo, c->node64, c->node32, c->hdr64, c->hdr32, d_cint,
                                              c->d_status);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(cint.data(), d_cint, 3 * N * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(d_cint);
        if (e != cudaSuccess) return set_err(c, BEM_ERR_CUDA, "P1 geometry: %s", cudaGetErrorString(e));
        ++c->cnt.kernel_launches;
    }
    int st = 0;
    BEM_CUDA_TRY(c, cudaMemcpy(&st, c->d_status, sizeof st, cudaMemcpyDeviceToHost));
    if (st) return set_err(c, BEM_ERR_DEGENERATE, "P1: a triangle's corners are collinear");
    k_chunk_spheres<<<nblk((N + 31) / 32, 128), 128, 0, s>>>(N, c->geo, c->chunk_sph);
    BEM_LAUNCH_CHECK(c);
    k_p1_targets<<<nblk(nv, 256), 256, 0, s>>>(D, c->tgt64, c->tgt32);
    BEM_LAUNCH_CHECK(c);
    // near pairs of the vertices (CSR)
    {
        int32_t* d_count = nullptr;
        if ((rc = p1_alloc(c, &d_count, nv)) || (rc = p1_alloc(c, &D.ptr, nv + 1))) {
            if (d_count) cudaFree(d_count);
            return rc;
        }
        k_p1_near_rows<<<nblk(nv * 32, 128), 128, 0, s>>>(D, 0, c->tgt32, c->tgt64, c->hdr32, c->hdr64, d_count,
                                                          nullptr, nullptr, nullptr);
        cudaError_t e = cudaGetLastError();
        std::vector<int32_t> cnt(nv);
        if (e == cudaSuccess) e = cudaMemcpyAsync(cnt.data(), d_count, nv * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFree(d_count);
        if (e != cudaSuccess) return set_err(c, BEM_ERR_CUDA, "P1 near pairs: %s", cudaGetErrorString(e));
        std::vector<int64_t> ptr(nv + 1, 0);
        for (int64_t v = 0; v < nv; ++v) ptr[v + 1] = ptr[v] + cnt[v];
        D.nnz = ptr[nv];
        c->nnz = D.nnz;
        if ((rc = p1_alloc(c, &D.col, D.nnz)) || (rc = p1_alloc(c, &D.flag, D.nnz)) ||
            (rc = p1_alloc(c, &D.val, 3 * D.nnz)))
            return rc;
        BEM_CUDA_TRY(c, cudaMemcpyAsync(D.ptr, ptr.data(), (nv + 1) * 8, cudaMemcpyHostToDevice, s));
        k_p1_near_rows<<<nblk(nv * 32, 128), 128, 0, s>>>(D, 1, c->tgt32, c->tgt64, c->hdr32, c->hdr64, nullptr,
                                                          D.ptr, D.col, D.flag);
        BEM_LAUNCH_CHECK(c);
        k_p1_near_values<<<nblk(D.nnz * 32, 128), 128, 0, s>>>(D, D.ptr, D.col, D.flag, D.val);
        BEM_LAUNCH_CHECK(c);
        std::vector<uint8_t> fl(D.nnz);
        BEM_CUDA_TRY(c, cudaMemcpyAsync(fl.data(), D.flag, D.nnz, cudaMemcpyDeviceToHost, s));
        BEM_CUDA_TRY(c, cudaStreamSynchronize(s));
        for (uint8_t f : fl) {
            c->nnz_prec[BEM_MIXED] += (f & 1) ? 1 : 0;
            c->nnz_prec[BEM_FP64] += (f & 2) ? 1 : 0;
        }
    }
    if ((rc = p1_dielectric_setup(c, nodes, tri6, vkind, vreg))) return rc;
    // neutrality weights a_f[v] = int_body psi_v dS (per corner, summed in triangle order)
    {
        std::vector<double> nw((size_t)std::max(c->nfloat, 1) * nv, 0.0);
        for (int64_t T = 0; T < N; ++T) {
            const bem_region& R = c->regions[region[T]];
            if (R.kind != BEM_FLOATING) continue;
            for (int k = 0; k < 3; ++k) nw[(size_t)R.floating_id * nv + tri6[6 * T + k]] += cint[3 * T + k];
        }
        if ((rc = p1_alloc(c, &D.neut_w, nw.size()))) return rc;
        BEM_CUDA_TRY(c, cudaMemcpyAsync(D.neut_w, nw.data(), nw.size() * 8, cudaMemcpyHostToDevice, s));
        BEM_CUDA_TRY(c, cudaStreamSynchronize(s));
    }
    // conductor potentials per region, Jacobi scaling, workspace
    const int nreg = (int)c->regions.size();
    std::vector<double> V0(nreg, 0.0);
    for (int r = 0; r < nreg; ++r) V0[r] = c->regions[r].kind == BEM_CONDUCTOR ? c->regions[r].V0 : 0.0;
    c->nunk = nv + c->nfloat;
    const int64_t n = c->nunk;
    if ((rc = p1_alloc(c, &c->region_V0, nreg)) || (rc = p1_alloc(c, &c->jinv, n))) return rc;
    BEM_CUDA_TRY(c, cudaMemcpyAsync(c->region_V0, V0.data(), nreg * 8, cudaMemcpyHostToDevice, s));
    k_p1_jacobi<<<nblk(n, 256), 256, 0, s>>>(D, n, c->jinv);
    BEM_LAUNCH_CHECK(c);
    size_t need = 0;
    for (int prec = 0; prec < 2; ++prec)
        for (int64_t M : {nv, (int64_t)c->prm.max_points, 4 * D.nd})
            need = std::max(need, (size_t)far_splits(c, prec, M) * (size_t)M * 4);
    c->part_cap = need;
    c->m = c->prm.gmres_restart;
    if ((rc = p1_alloc(c, &c->part, need)) || (rc = p1_alloc(c, &c->V, (size_t)(c->m + 1) * n)) ||
        (rc = p1_alloc(c, &c->wvec, n)) || (rc = p1_alloc(c, &c->zvec, n)) || (rc = p1_alloc(c, &c->rvec, n)) ||
        (rc = p1_alloc(c, &c->bvec, n)) || (rc = p1_alloc(c, &c->dvec, n)) || (rc = p1_alloc(c, &c->ivec, n)) ||
        (rc = p1_alloc(c, &c->hcol, 2 * (c->m + 2))))
        return rc;
    if (cudaMallocHost((void**)&c->hcol_host, 2 * (c->m + 2) * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        c->hcol_host = nullptr;
        return set_err(c, BEM_ERR_NOMEM, "cudaMallocHost failed");
    }
    if (c->prm.timing) {
        const int pool = 1024;
        c->ev0.resize(pool);
        c->ev1.resize(pool);
        c->ev_prec.assign(pool, 0);
        for (int k = 0; k < pool; ++k) {
            BEM_CUDA_TRY(c, cudaEventCreate(&c->ev0[k]));
            BEM_CUDA_TRY(c, cudaEventCreate(&c->ev1[k]));
        }
    }
    c->tune.far32_variant = c->far32_tp;
    c->tune.far32_slots = c->far_slots;
    c->cnt = bem_counters{};
    c->cnt.far32_variant = c->far32_tp;
    BEM_CUDA_TRY(c, cudaStreamSynchronize(s));
    return BEM_OK;
}

extern "C" int bem_p1_create(bem_ctx** out, int64_t nn, const double* nodes, int64_t nv, int64_t N,
                             const int32_t* tri6, const int32_t* region, int32_t nregions,
                             const bem_region* regions, const bem_p1_params* params, void* stream)
{
    if (!out) return set_err(nullptr, BEM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!nodes || !tri6 || !region || !regions || nn < 3 || nv < 3 || nv > nn || N < 1 || nregions < 1 ||
        N > ((int64_t)1 << 28))
        return set_err(nullptr, BEM_ERR_ARG, "bem_p1_create: bad sizes or NULL arrays");
    bem_p1_params p;
    if (params) p = *params;
    else bem_p1_default_params(&p);
    if (!(p.eta >= 1.0) || p.far_order < 1 || p.far_order > kMaxOrder || p.sing_order < 1 || p.sing_order > 64 ||
        p.near_radial < 1 || p.near_radial > 64 || p.near_angular < 1 || p.near_angular > 256 ||
        p.gmres_restart < 1 || p.gmres_restart > 1000 || p.max_iters < 1 || p.max_refine < 1 ||
        p.max_points < 1 || p.far32_variant < 2 || p.far32_variant > 4)
        return set_err(nullptr, BEM_ERR_ARG, "bem_p1_create: bad parameters");
    for (int64_t i = 0; i < 6 * N; ++i)
        if (tri6[i] < 0 || tri6[i] >= nn || (i % 6 < 3 && tri6[i] >= nv))
            return set_err(nullptr, BEM_ERR_ARG, "bem_p1_create: node index out of range in triangle %lld",
                           (long long)(i / 6));
    int nfloat = 0;
    for (int r = 0; r < nregions; ++r) {
        const bem_region& R = regions[r];
        if (R.kind != BEM_CONDUCTOR && R.kind != BEM_FLOATING && R.kind != BEM_DIELECTRIC)
            return set_err(nullptr, BEM_ERR_ARG, "bem_p1_create: region %d: only conductor, floating and "
                           "dielectric regions are built on the curved-triangle path", r);
        if (R.kind == BEM_FLOATING) nfloat = std::max(nfloat, R.floating_id + 1);
    }
    for (int64_t T = 0; T < N; ++T)
        if (region[T] < 0 || region[T] >= nregions)
            return set_err(nullptr, BEM_ERR_ARG, "bem_p1_create: region index out of range");
    bem_ctx* c = new (std::nothrow) bem_ctx();
    if (!c) return set_err(nullptr, BEM_ERR_NOMEM, "out of host memory");
    c->stream = (cudaStream_t)stream;
    cudaGetDevice(&c->device);
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    bem_default_params(&c->prm);
    c->prm.eta = p.eta;
    c->prm.far_order = p.far_order;
    c->prm.gmres_restart = p.gmres_restart;
    c->prm.max_iters = p.max_iters;
    c->prm.max_refine = p.max_refine;
    c->prm.max_points = p.max_points;
    c->prm.timing = p.timing;
    c->prm.residual = BEM_RESIDUAL_FP64;   // the refinement residual: the FP64 kernel
    c->prm.far32_variant = p.far32_variant;
    c->prm.adjoint_lines = 0;
    c->regions.assign(regions, regions + nregions);
    c->h_region.assign(region, region + N);
    c->nfloat = nfloat;
    int rc = p1_create_impl(c, nn, nodes, nv, N, tri6, region, p);
    if (rc) {
        const std::string msg = c->err;
        bem_destroy(c);
        return set_err(nullptr, rc, "%s", msg.c_str());
    }
    *out = c;
    return BEM_OK;
}

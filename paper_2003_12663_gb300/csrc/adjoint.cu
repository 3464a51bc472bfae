// adjoint.cu -- gradient of J = sum_l w_l K_l (K_l the breakdown integral of
// Eq. Breakdowncrit along line l) with respect to the vertex coordinates, the
// conductor potentials V0 and the permittivities, through the solve of Eqs.
// Final1-Final4 and the field-line integration.  Not in the paper; it makes K a
// differentiable design objective.
//
// Discrete adjoint of exactly what bem_solve + bem_trace_lines compute:
//   dJ/dtheta = dJ/dtheta|_u + mu^T (db/dtheta - dA/dtheta u),   A^T mu = dJ/du.
// 1. Forward again with a tape: every step's start state and its sub-steps
//    (lengths and event kinds), from the same integrator as bem_trace_lines.
// 2. Reverse sweep per line (one CTA per line): every sub-step is recomputed with
//    the field Jacobian at its four stages; the RK4 step is differentiated in
//    reverse; a located crossing contributes through the implicit function
//    theorem, d sigma* = -(dg/dtheta)/(dg/dsigma), with dg/dsigma from a forward
//    tangent of the re-stepped RK4 step.  Each stage's field cotangent lam_E is
//    pushed into dJ/du_j = lam_E.G_j(y) and into the triangles' vertex gradients.
// 3. A^T mu = dJ/du by GMRES on the transposed operator (point charges and
//    dipoles at the centroids, integrated over every triangle).
// 4. -mu^T (dA/dX) u pair by pair (target side: centroid, normal and area of row
//    i; source side: vertices of triangle j), V0 and eps gradients per region.
// Regular pairs are differentiated in closed form on the Duffy/Gauss nodes; near
// pairs by forward-mode dual numbers through the closed-form integral.
#include <algorithm>
#include <vector>

#include "dual.cuh"
#include "trace_core.cuh"

int trace_args(bem_ctx* c, const bem_trace_params* tp, const double* u, tcore::TArgs* out);
int solve_transpose(bem_ctx* c, int precision, const double* rhs, double* x, double tol, int* iters,
                    double* relres);

namespace {

using namespace tcore;

__constant__ double c_ru[kMaxOrder], c_rv[kMaxOrder];  // node (u_k, v_l) of the Duffy rule

struct StepRec {
    double x[3];
    double K;
    double sig[4];
    int32_t side;
    int32_t nsub;
    int32_t kind[4];
};

// The state of a line at the start of a step: what a resumed trace starts from.
struct Ckpt {
    double x[3];
    double K;
    int32_t side;
    int32_t pad;
};

// Forward recorder: the state at the start of every k-th step (checkpoints) and the
// number of step records the line produces.
struct CkptRec {
    Ckpt* cp;
    int64_t ncp;
    int k;
    int64_t n;
    double s0;
    int seed_region;
    __device__ void begin(double s, int sr) { s0 = s; seed_region = sr; }
    __device__ void step(int64_t st, const double* x, double K, int side)
    {
        n = st + 1;
        if (st % k == 0 && st / k < ncp && (threadIdx.x & 31) == 0) {
            Ckpt& c = cp[st / k];
            c.x[0] = x[0]; c.x[1] = x[1]; c.x[2] = x[2];
            c.K = K;
            c.side = side;
        }
    }
    __device__ void sub(int64_t, int, double, int) {}
};

// Segment recorder: the step records (start state and sub-steps) of steps
// [step0, step0 + k), from a resumed trace.
struct SegRec {
    StepRec* tape;
    int64_t step0;
    int k;
    __device__ void begin(double, int) {}
    __device__ void step(int64_t st, const double* x, double K, int side)
    {
        const int64_t i = st - step0;
        if (i >= 0 && i < k && (threadIdx.x & 31) == 0) {
            StepRec& r = tape[i];
            r.x[0] = x[0]; r.x[1] = x[1]; r.x[2] = x[2];
            r.K = K;
            r.side = side;
            r.nsub = 0;
        }
    }
    __device__ void sub(int64_t st, int kk, double sig, int kind)
    {
        const int64_t i = st - step0;
        if (i >= 0 && i < k && kk < 4 && (threadIdx.x & 31) == 0) {
            tape[i].sig[kk] = sig;
            tape[i].kind[kk] = kind;
            tape[i].nsub = kk + 1;
        }
    }
};

// forward with checkpoints: the persistent tracer launch of bem_trace_lines with a
// checkpoint recorder per line (cp: [L][ncp])
template <bool F32, int Q>
__global__ void __launch_bounds__(kLT)
k_adj_forward(TArgs A, const double* __restrict__ seeds, int64_t L, unsigned long long* __restrict__ next,
              Ckpt* __restrict__ cp, int64_t ncp, int k, int64_t* __restrict__ nrec,
              double* __restrict__ s0_out, int* __restrict__ sr_out, double* __restrict__ K_out,
              int32_t* __restrict__ st_out)
{
    __shared__ Round R;
    __shared__ TArgs sA;
    __shared__ int s_int[3];
    run_lines<F32, Q>([&](int) { return A; }, [&](int) { return L; }, 1, L, next, sA, R, s_int,
                      [&](const TArgs& a, Round& r, int, int64_t line) {
                          CkptRec rec{cp + line * ncp, ncp, k, 0, 1.0, -1};
                          double K, xe[3];
                          int st;
                          int64_t ns;
                          trace_line<F32, Q>(a, r, seeds + 3 * line, rec, K, st, ns, xe);
                          if ((threadIdx.x & 31) == 0) {
                              nrec[line] = rec.n;
                              s0_out[line] = rec.s0;
                              sr_out[line] = rec.seed_region;
                              K_out[line] = K;
                              st_out[line] = st;
                          }
                      });
}

// segment seg of every line: resume from checkpoint seg and record steps
// [seg k, seg k + k) into tape[line][0..k); segn[line] = records written
template <bool F32, int Q>
__global__ void __launch_bounds__(kLT)
k_adj_resume(TArgs A, int64_t L, unsigned long long* __restrict__ next, const Ckpt* __restrict__ cp,
             int64_t ncp, int k, int64_t seg, const int64_t* __restrict__ nrec,
             const double* __restrict__ s0s, const int* __restrict__ srs, StepRec* __restrict__ tape,
             int64_t* __restrict__ segn)
{
    __shared__ Round R;
    __shared__ TArgs sA;
    __shared__ int s_int[3];
    run_lines<F32, Q>([&](int) { return A; }, [&](int) { return L; }, 1, L, next, sA, R, s_int,
                      [&](const TArgs& a, Round& r, int, int64_t line) {
                          const int64_t n = nrec[line], st0 = seg * (int64_t)k;
                          if (n <= st0) {
                              if ((threadIdx.x & 31) == 0) segn[line] = 0;
                              return;
                          }
                          const Ckpt c = cp[line * ncp + seg];
                          double x[3] = {c.x[0], c.x[1], c.x[2]};
                          double K = c.K;
                          SegRec rec{tape + line * (int64_t)k, st0, k};
                          int st;
                          int64_t ns;
                          trace_steps<F32, Q>(a, r, x, K, c.side, s0s[line], srs[line], st0, st0 + k, rec, st, ns);
                          if ((threadIdx.x & 31) == 0) segn[line] = min(n, st0 + k) - st0;
                      });
}

// ---------------------------------------------------------------- CTA passes
// CTA sums of NV values in a fixed order, returned to every thread: warp butterflies,
// then lane i adds value i over the warps (in warp order) and shuffles it to all lanes
template <int NV>
__device__ void block_sum_n(double* v, double* sh)
{
    static_assert(NV <= 32, "one lane per value");
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = wsum(v[i]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) sh[i * kWarps + warp] = v[i];
    __syncthreads();
    const int li = min(lane, NV - 1);
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s += sh[li * kWarps + w];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = __shfl_sync(0xffffffffu, s, i);
}

// E(x) and its Jacobian J = dE/dx (symmetric: xx, yy, zz, xy, xz, yz) -> out[9]
template <bool F32, int Q>
__device__ __noinline__ void cta_field_jac(const TArgs& A, const double* x, double* out, double* sh)
{
    const float xf = __double2float_rn(x[0]), yf = __double2float_rn(x[1]), zf = __double2float_rn(x[2]);
    float f[9];
    double q[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) { f[i] = 0.f; q[i] = 0.0; }
    for (int64_t j = threadIdx.x; j < A.np; j += kT) {
        const double uj = A.u[j];
        const double* gp = A.geo + GEO_STRIDE * j;
        const bool far = F32 ? is_far32(xf, yf, zf, A.hdr32[j]) : is_far64(x[0], x[1], x[2], A.hdr64[j]);
        if (far && F32) {
            float g[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) g[i] = 0.f;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const float4 nd = A.node32[j * Q + k];
                const float dx = xf - nd.x, dy = yf - nd.y, dz = zf - nd.z;
                const float ri = rsqrtf(dx * dx + dy * dy + dz * dz);
                const float ri2 = ri * ri, w3 = nd.w * ri * ri2, t = 3.f * ri2;
                g[0] += w3 * dx; g[1] += w3 * dy; g[2] += w3 * dz;
                g[3] += w3 * (1.f - t * dx * dx); g[4] += w3 * (1.f - t * dy * dy); g[5] += w3 * (1.f - t * dz * dz);
                g[6] -= w3 * t * dx * dy; g[7] -= w3 * t * dx * dz; g[8] -= w3 * t * dy * dz;
            }
            const float uf = __double2float_rn(uj);
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = fmaf(uf, g[i], f[i]);
        } else if (far) {
            double g[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) g[i] = 0.0;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const double4 nd = A.node64[j * Q + k];
                const double dx = x[0] - nd.x, dy = x[1] - nd.y, dz = x[2] - nd.z;
                const double ri = rsqrt(dx * dx + dy * dy + dz * dz);
                const double ri2 = ri * ri, w3 = nd.w * ri * ri2, t = 3.0 * ri2;
                g[0] += w3 * dx; g[1] += w3 * dy; g[2] += w3 * dz;
                g[3] += w3 * (1.0 - t * dx * dx); g[4] += w3 * (1.0 - t * dy * dy); g[5] += w3 * (1.0 - t * dz * dz);
                g[6] -= w3 * t * dx * dy; g[7] -= w3 * t * dx * dz; g[8] -= w3 * t * dy * dz;
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) q[i] = fma(uj, g[i], q[i]);
        } else {
            Dual<3> xd[3] = {dvar<3>(x[0], 0), dvar<3>(x[1], 1), dvar<3>(x[2], 2)};
            Dual<3> vd[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) vd[i] = dconst<3>(gp[i]);
            Dual<3> S, G[3];
            tri_cf_t<Dual<3>>(vd, xd, false, S, G);
            // closed-form values carry 1/(4 pi) already; rescale to the quadrature's units
            const double s = uj * (4.0 * M_PI);
            q[0] += s * G[0].v; q[1] += s * G[1].v; q[2] += s * G[2].v;
            q[3] += s * G[0].d[0]; q[4] += s * G[1].d[1]; q[5] += s * G[2].d[2];
            q[6] += s * 0.5 * (G[0].d[1] + G[1].d[0]);
            q[7] += s * 0.5 * (G[0].d[2] + G[2].d[0]);
            q[8] += s * 0.5 * (G[1].d[2] + G[2].d[1]);
        }
    }
    double v[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) v[i] = kInv4Pi * (q[i] + (double)f[i]);
    block_sum_n<9>(v, sh);
    // reorder to E[3], J[6] = (xx, yy, zz, xy, xz, yz)
#pragma unroll
    for (int i = 0; i < 9; ++i) out[i] = v[i];
}

__device__ __forceinline__ void area_grad(const double* gp, double* dA)  // dA/d(a,b,c), 9 values
{
    const double nx = gp[GEO_N], ny = gp[GEO_N + 1], nz = gp[GEO_N + 2];
    const double* v = gp;
    // dA/da = n x (c - b) / 2, dA/db = n x (a - c) / 2, dA/dc = n x (b - a) / 2
    for (int corner = 0; corner < 3; ++corner) {
        const int p = (corner + 1) % 3, q = (corner + 2) % 3;  // (c - b) for a: q = c, p = b
        const double ex = v[3 * q] - v[3 * p], ey = v[3 * q + 1] - v[3 * p + 1], ez = v[3 * q + 2] - v[3 * p + 2];
        dA[3 * corner] = 0.5 * (ny * ez - nz * ey);
        dA[3 * corner + 1] = 0.5 * (nz * ex - nx * ez);
        dA[3 * corner + 2] = 0.5 * (nx * ey - ny * ex);
    }
}

// Contracted derivatives of F = kS S_j(x) + kG.G_j(x) (regular pair, Duffy/Gauss
// nodes of triangle j): value, dF/dx (3), dF/d(a,b,c) (9).  T: float or double.
template <class T, int Q>
__device__ __forceinline__ void far_pair_grad(const double* gp, const float4* n32, const double4* n64,
                                              int64_t j, int g, const double* x, double kS,
                                              const double* kG, bool want_x, bool want_v, double& F,
                                              double* dx_out, double* dv_out)
{
    T Fv = 0, fx[3] = {0, 0, 0}, gv[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) gv[i] = 0;
    const T xs[3] = {(T)x[0], (T)x[1], (T)x[2]};
    const T ks = (T)kS, kg[3] = {(T)kG[0], (T)kG[1], (T)kG[2]};
#pragma unroll
    for (int k = 0; k < Q; ++k) {
        T yx, yy, yz, w;
        if (sizeof(T) == 4) {
            const float4 nd = n32[j * Q + k];
            yx = nd.x; yy = nd.y; yz = nd.z; w = nd.w;
        } else {
            const double4 nd = n64[j * Q + k];
            yx = (T)nd.x; yy = (T)nd.y; yz = (T)nd.z; w = (T)nd.w;
        }
        const T dx = xs[0] - yx, dy = xs[1] - yy, dz = xs[2] - yz;
        const T ri = (T)1 / sqrt(dx * dx + dy * dy + dz * dz);
        const T ri2 = ri * ri, ri3 = ri * ri2;
        const T kd = kg[0] * dx + kg[1] * dy + kg[2] * dz;
        Fv += w * (ks * ri + kd * ri3);
        // d/dx of w (ks/r + kG.d/r^3)
        const T c1 = w * (-ks * ri3 - (T)3 * kd * ri3 * ri2), c2 = w * ri3;
        const T gx = c1 * dx + c2 * kg[0], gy = c1 * dy + c2 * kg[1], gz = c1 * dz + c2 * kg[2];
        fx[0] += gx; fx[1] += gy; fx[2] += gz;
        if (want_v) {
            const int kk = k / g, ll = k % g;
            const T u = (T)c_ru[kk], v = (T)c_rv[ll];
            const T al = (T)1 - u, be = u * ((T)1 - v), ga = u * v;  // y = al a + be b + ga c
            gv[0] -= al * gx; gv[1] -= al * gy; gv[2] -= al * gz;
            gv[3] -= be * gx; gv[4] -= be * gy; gv[5] -= be * gz;
            gv[6] -= ga * gx; gv[7] -= ga * gy; gv[8] -= ga * gz;
        }
    }
    F = kInv4Pi * (double)Fv;
    if (want_x)
        for (int c = 0; c < 3; ++c) dx_out[c] = kInv4Pi * (double)fx[c];
    if (want_v) {
        double dA[9];
        area_grad(gp, dA);
        const double Fa = F / gp[GEO_AREA];  // weights scale with the area
        for (int i = 0; i < 9; ++i) dv_out[i] = kInv4Pi * (double)gv[i] + Fa * dA[i];
    }
}

// Near pair: the same contracted derivatives through the closed form.  which: 0
// -> d/dx (x seeded), 1 -> d/d(a,b,c) (vertices seeded).
__device__ __noinline__ void near_pair_grad(const double* gp, const double* x, bool own, double kS,
                                            const double* kG, int which, double& F, double* d)
{
    if (which == 0) {
        Dual<3> xd[3] = {dvar<3>(x[0], 0), dvar<3>(x[1], 1), dvar<3>(x[2], 2)};
        Dual<3> vd[9];
        for (int i = 0; i < 9; ++i) vd[i] = dconst<3>(gp[i]);
        Dual<3> S, G[3];
        tri_cf_t<Dual<3>>(vd, xd, own, S, G);
        F = kS * S.v + kG[0] * G[0].v + kG[1] * G[1].v + kG[2] * G[2].v;
        for (int c = 0; c < 3; ++c) d[c] = kS * S.d[c] + kG[0] * G[0].d[c] + kG[1] * G[1].d[c] + kG[2] * G[2].d[c];
    } else {
        Dual<9> vd[9], xd[3];
        for (int i = 0; i < 9; ++i) vd[i] = dvar<9>(gp[i], i);
        if (own) {  // the target is the triangle's own centroid: it moves with the vertices
            for (int c = 0; c < 3; ++c) xd[c] = (1.0 / 3.0) * (vd[c] + vd[3 + c] + vd[6 + c]);
        } else {
            for (int c = 0; c < 3; ++c) xd[c] = dconst<9>(x[c]);
        }
        Dual<9> S, G[3];
        tri_cf_t<Dual<9>>(vd, xd, own, S, G);
        F = kS * S.v + kG[0] * G[0].v + kG[1] * G[1].v + kG[2] * G[2].v;
        for (int i = 0; i < 9; ++i) d[i] = kS * S.d[i] + kG[0] * G[0].d[i] + kG[1] * G[1].d[i] + kG[2] * G[2].d[i];
    }
}

// Push a field cotangent lam (at point y) into dJ/du_j += lam.G_j(y) and the
// vertex gradients u_j d(lam.G_j(y))/d(a,b,c); each thread owns its triangles.
template <bool F32, int Q>
__device__ __noinline__ void cta_record(const TArgs& A, int g, const double* y, const double* lam,
                                        double* gu, double* gp_out)
{
    const float yf = __double2float_rn(y[0]), yyf = __double2float_rn(y[1]), yzf = __double2float_rn(y[2]);
    for (int64_t j = threadIdx.x; j < A.np; j += kT) {
        const double uj = A.u[j];
        const double* gp = A.geo + GEO_STRIDE * j;
        const bool far = F32 ? is_far32(yf, yyf, yzf, A.hdr32[j]) : is_far64(y[0], y[1], y[2], A.hdr64[j]);
        double F, dv[9];
        if (far) {
            if (F32)
                far_pair_grad<float, Q>(gp, A.node32, A.node64, j, g, y, 0.0, lam, false, true, F, nullptr, dv);
            else
                far_pair_grad<double, Q>(gp, A.node32, A.node64, j, g, y, 0.0, lam, false, true, F, nullptr, dv);
        } else {
            near_pair_grad(gp, y, false, 0.0, lam, 1, F, dv);
        }
        gu[j] += F;
        for (int i = 0; i < 9; ++i) gp_out[9 * j + i] += uj * dv[i];
    }
}

// ---------------------------------------------------------------- reverse sweep
struct Stage {
    double y[3], E[3], J[6];
};

__device__ __forceinline__ void jmul(const double* J, const double* v, double* o)
{
    o[0] = J[0] * v[0] + J[3] * v[1] + J[4] * v[2];
    o[1] = J[3] * v[0] + J[1] * v[1] + J[5] * v[2];
    o[2] = J[4] * v[0] + J[5] * v[1] + J[2] * v[2];
}

template <bool F32, int Q>
__global__ void __launch_bounds__(kT)
k_adj_backward(TArgs A, int g, const StepRec* __restrict__ tape, int k, const int64_t* __restrict__ segn,
               const double* __restrict__ s0s, const double* __restrict__ wts, int64_t nl,
               double* __restrict__ gu_l, double* __restrict__ gp_l, double* __restrict__ lx_l)
{
    __shared__ double sh[9 * kWarps];
    __shared__ Stage s_st[4][4];
    __shared__ double s_ev[4][12];  // end point (3), and at a crossing E (3) and J (6)
    __shared__ double s_xs[4][4];  // sub-step start x (3) and K
    // one segment of one line per CTA: the line's gradient buffers and the adjoint of
    // its state (lx) carry over from the later segments, reversed before this one
    const int64_t b = blockIdx.x;
    if (b >= nl) return;
    double* gu = gu_l + b * A.np;
    double* gpv = gp_l + b * A.np * 9;
    const double s0 = s0s[b];
    const double lamK = wts[b];
    double lx[3] = {lx_l[3 * b], lx_l[3 * b + 1], lx_l[3 * b + 2]};
    const StepRec* tp = tape + b * (int64_t)k;
    const double cw[4] = {1.0, 2.0, 2.0, 1.0};
    for (int64_t r = segn[b] - 1; r >= 0; --r) {
        const StepRec R = tp[r];
        // recompute the sub-steps with field Jacobians at their stages
        double xs[3] = {R.x[0], R.x[1], R.x[2]}, Ks = R.K;
        int side = R.side;
        int sides[4];
        for (int k = 0; k < R.nsub; ++k) {
            sides[k] = side;
            const double sg = R.sig[k];
            double kv[4][3], a[4];
            for (int st = 0; st < 4; ++st) {
                double y[3];
                for (int c = 0; c < 3; ++c)
                    y[c] = st == 0 ? xs[c] : xs[c] + kv[st - 1][c] * (st < 3 ? 0.5 * sg : sg);
                double o[9];
                cta_field_jac<F32, Q>(A, y, o, sh);
                const double Em = norm3(o[0], o[1], o[2]);
                for (int c = 0; c < 3; ++c) kv[st][c] = o[c] * (s0 / Em);
                a[st] = alpha_eff(A, Em, side);
                if (threadIdx.x == 0) {
                    Stage& S = s_st[k][st];
                    for (int c = 0; c < 3; ++c) { S.y[c] = y[c]; S.E[c] = o[c]; }
                    for (int c = 0; c < 6; ++c) S.J[c] = o[3 + c];
                }
            }
            if (threadIdx.x == 0) { s_xs[k][0] = xs[0]; s_xs[k][1] = xs[1]; s_xs[k][2] = xs[2]; s_xs[k][3] = Ks; }
            for (int c = 0; c < 3; ++c) xs[c] += ((kv[0][c] + (kv[1][c] + kv[2][c]) * 2.0) + kv[3][c]) * (sg / 6.0);
            Ks += sg / 6.0 * (a[0] + 2.0 * (a[1] + a[2]) + a[3]);
            if (threadIdx.x == 0) { s_ev[k][0] = xs[0]; s_ev[k][1] = xs[1]; s_ev[k][2] = xs[2]; }
            if (R.kind[k] == SUB_ALPHA) {  // field and Jacobian at the crossing
                double o[9];
                cta_field_jac<F32, Q>(A, xs, o, sh);
                if (threadIdx.x == 0)
                    for (int c = 0; c < 9; ++c) s_ev[k][3 + c] = o[c];
                side = -side;
            }
        }
        __syncthreads();
        // reverse over the sub-steps
        double lrem = 0.0;
        for (int k = R.nsub - 1; k >= 0; --k) {
            const double sg = R.sig[k];
            const int sd = sides[k];
            double Em[4], e[4][3], kv[4][3], a[4], ap[4];
            for (int st = 0; st < 4; ++st) {
                const Stage& S = s_st[k][st];
                Em[st] = norm3(S.E[0], S.E[1], S.E[2]);
                for (int c = 0; c < 3; ++c) { e[st][c] = S.E[c] / Em[st]; kv[st][c] = s0 * e[st][c]; }
                a[st] = alpha_eff(A, Em[st], sd);
                ap[st] = sd > 0 ? 2.0 * A.c * (Em[st] - A.E0) : 0.0;
            }
            double seed[3] = {lx[0], lx[1], lx[2]};
            const int kind = R.kind[k];
            double gam = 0.0, ge[3] = {0.0, 0.0, 0.0};
            if (kind == SUB_ALPHA || kind == SUB_RMAX) {
                // forward tangent of the sub-step's end w.r.t. its length
                double kd[4][3] = {{0, 0, 0}}, ad[4] = {0, 0, 0, 0};
                for (int st = 1; st < 4; ++st) {
                    const double fd = st < 3 ? 0.5 : 1.0, f = st < 3 ? 0.5 * sg : sg;
                    double yd[3], Ed[3];
                    for (int c = 0; c < 3; ++c) yd[c] = fd * kv[st - 1][c] + f * kd[st - 1][c];
                    jmul(s_st[k][st].J, yd, Ed);
                    const double eE = e[st][0] * Ed[0] + e[st][1] * Ed[1] + e[st][2] * Ed[2];
                    for (int c = 0; c < 3; ++c) kd[st][c] = s0 / Em[st] * (Ed[c] - e[st][c] * eE);
                    ad[st] = ap[st] * eE;
                }
                double xd[3], Kd;
                for (int c = 0; c < 3; ++c)
                    xd[c] = (kv[0][c] + 2.0 * (kv[1][c] + kv[2][c]) + kv[3][c]) / 6.0 +
                            sg / 6.0 * (kd[0][c] + 2.0 * (kd[1][c] + kd[2][c]) + kd[3][c]);
                Kd = (a[0] + 2.0 * (a[1] + a[2]) + a[3]) / 6.0 + sg / 6.0 * (ad[0] + 2.0 * (ad[1] + ad[2]) + ad[3]);
                // dg/dx at the end point
                if (kind == SUB_ALPHA) {  // g = |E(x_e)| - E0: dg/dx = J e
                    const double* o = s_ev[k] + 3;
                    const double Ee = norm3(o[0], o[1], o[2]);
                    const double ee[3] = {o[0] / Ee, o[1] / Ee, o[2] / Ee};
                    jmul(o + 3, ee, ge);
                } else {  // g = |x_e| - r_max
                    const double* xe = s_ev[k];
                    const double re = norm3(xe[0], xe[1], xe[2]);
                    for (int c = 0; c < 3; ++c) ge[c] = xe[c] / re;
                }
                const double gdot = ge[0] * xd[0] + ge[1] * xd[1] + ge[2] * xd[2];
                const double lsig = lx[0] * xd[0] + lx[1] * xd[1] + lx[2] * xd[2] + lamK * Kd - lrem;
                gam = -lsig / gdot;
                for (int c = 0; c < 3; ++c) seed[c] += gam * ge[c];
            }
            // reverse RK4 of this sub-step with cotangents (seed, lamK)
            double lk[4][3], la[4], lxs[3] = {seed[0], seed[1], seed[2]};
            double lsg = 0.0;
            for (int st = 0; st < 4; ++st) {
                for (int c = 0; c < 3; ++c) lk[st][c] = seed[c] * sg / 6.0 * cw[st];
                la[st] = lamK * sg / 6.0 * cw[st];
                lsg += cw[st] / 6.0 * (seed[0] * kv[st][0] + seed[1] * kv[st][1] + seed[2] * kv[st][2] + lamK * a[st]);
            }
            for (int st = 3; st >= 0; --st) {
                const double el = e[st][0] * lk[st][0] + e[st][1] * lk[st][1] + e[st][2] * lk[st][2];
                double lE[3];
                for (int c = 0; c < 3; ++c) lE[c] = s0 / Em[st] * (lk[st][c] - e[st][c] * el) + ap[st] * e[st][c] * la[st];
                cta_record<F32, Q>(A, g, s_st[k][st].y, lE, gu, gpv);
                double ly[3];
                jmul(s_st[k][st].J, lE, ly);
                for (int c = 0; c < 3; ++c) lxs[c] += ly[c];
                if (st > 0) {
                    const double f = st < 3 ? 0.5 * sg : sg, fd = st < 3 ? 0.5 : 1.0;
                    for (int c = 0; c < 3; ++c) lk[st - 1][c] += f * ly[c];
                    lsg += fd * (ly[0] * kv[st - 1][0] + ly[1] * kv[st - 1][1] + ly[2] * kv[st - 1][2]);
                }
            }
            if (kind == SUB_ALPHA) {  // g = |E(x_e)| - E0 also depends on the field directly
                const double* o = s_ev[k] + 3;
                const double Ee = norm3(o[0], o[1], o[2]);
                double lE[3];
                for (int c = 0; c < 3; ++c) lE[c] = gam * o[c] / Ee;
                cta_record<F32, Q>(A, g, s_ev[k], lE, gu, gpv);
            }
            if (kind == SUB_PLAIN) lrem += lsg;
            lx[0] = lxs[0]; lx[1] = lxs[1]; lx[2] = lxs[2];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        lx_l[3 * b] = lx[0];
        lx_l[3 * b + 1] = lx[1];
        lx_l[3 * b + 2] = lx[2];
    }
}

// sum the per-line buffers (fixed order)
__global__ void k_sum_lines(int64_t nl, int64_t n, const double* __restrict__ src, double* __restrict__ dst)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = dst[i];
    for (int64_t l = 0; l < nl; ++l) s += src[l * n + i];
    dst[i] = s;
}

// ---------------------------------------------------------------- transposed operator
// Sources of A^T v: row i carries a point charge alpha_i (conductor and floating
// rows) and a dipole beta_i (dielectric rows: (eps+ - eps-) v_i n_i; floating rows:
// the neutrality weight A_i eps+ / area_f times v_{N+f}, along n_i).
__global__ void k_tsrc(int64_t np, const int32_t* __restrict__ kind, const int32_t* __restrict__ aux,
                       const double* __restrict__ rb, const double* __restrict__ rw,
                       const double* __restrict__ geo, const double* __restrict__ v,
                       double4* __restrict__ src64, float4* __restrict__ src32)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    const double* gp = geo + GEO_STRIDE * i;
    double al = 0.0, be = 0.0;
    if (kind[i] == BEM_CONDUCTOR) {
        al = v[i];
    } else if (kind[i] == BEM_FLOATING) {
        al = v[i];
        be = rw[i] * v[np + aux[i]];
    } else {
        be = rb[i] * v[i];
    }
    const double4 s = make_double4(al, be * gp[GEO_N], be * gp[GEO_N + 1], be * gp[GEO_N + 2]);
    src64[i] = s;
    src32[i] = make_float4((float)s.x, (float)s.y, (float)s.z, (float)s.w);
}

// (A^T v)_j far part: sum over rows i with a regular pair (c_i, tau_j) of
// sum_k w_jk [alpha_i / |c_i - y_jk| + beta_i.(c_i - y_jk) / |c_i - y_jk|^3].
template <bool F32, int Q>
__global__ void __launch_bounds__(128)
k_far_T(int64_t np, const float4* __restrict__ t32, const double4* __restrict__ t64,
        const float4* __restrict__ hdr32, const double4* __restrict__ hdr64,
        const float4* __restrict__ n32, const double4* __restrict__ n64,
        const float4* __restrict__ s32, const double4* __restrict__ s64, int64_t per_split,
        double* __restrict__ part)
{
    constexpr int PC = 64;
    __shared__ double4 sp[PC], ss[PC];
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t jj = min(j, np - 1);
    const int64_t i0 = blockIdx.y * per_split, i1 = min(np, i0 + per_split);
    double acc = 0.0;
    float accf = 0.f;
    for (int64_t c0 = i0; c0 < i1; c0 += PC) {
        const int n = (int)min((int64_t)PC, i1 - c0);
        __syncthreads();
        for (int k = threadIdx.x; k < n; k += blockDim.x) {
            const double4 p = t64[c0 + k];
            sp[k] = p;
            ss[k] = s64[c0 + k];
        }
        __syncthreads();
        if (F32) {
            const float4 h = hdr32[jj];
            float pc = 0.f;
            for (int k = 0; k < n; ++k) {
                const float4 tp = t32[c0 + k];
                const float4 sv = s32[c0 + k];
                if (!is_far32(tp.x, tp.y, tp.z, h)) continue;
                float s = 0.f;
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const float4 nd = n32[jj * Q + q];
                    const float dx = tp.x - nd.x, dy = tp.y - nd.y, dz = tp.z - nd.z;
                    const float ri = rsqrtf(dx * dx + dy * dy + dz * dz);
                    s += nd.w * (sv.x * ri + (sv.y * dx + sv.z * dy + sv.w * dz) * ri * ri * ri);
                }
                pc += s;
            }
            accf += pc;
        } else {
            const double4 h = hdr64[jj];
            for (int k = 0; k < n; ++k) {
                const double4 tp = sp[k];
                if (!is_far64(tp.x, tp.y, tp.z, h)) continue;
                const double4 sv = ss[k];
                double s = 0.0;
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const double4 nd = n64[jj * Q + q];
                    const double dx = tp.x - nd.x, dy = tp.y - nd.y, dz = tp.z - nd.z;
                    const double ri = rsqrt(dx * dx + dy * dy + dz * dz);
                    s += nd.w * (sv.x * ri + (sv.y * dx + sv.z * dy + sv.w * dz) * ri * ri * ri);
                }
                acc += s;
            }
        }
    }
    if (j < np) part[blockIdx.y * np + j] = kInv4Pi * (acc + (double)accf);
}

// finish A^T v for columns j < N: far partials + near pairs (column list) +
// dielectric diagonal + the u_j terms of the neutrality rows (1/2, and a sheet's eps-)
__global__ void k_finish_T(int64_t np, int splits, const double* __restrict__ part,
                           const int64_t* __restrict__ cptr, const int32_t* __restrict__ crow,
                           const int64_t* __restrict__ cent, const double4* __restrict__ val,
                           const uint8_t* __restrict__ flag, uint8_t bit,
                           const double4* __restrict__ src, const int32_t* __restrict__ kind,
                           const int32_t* __restrict__ aux, const double* __restrict__ ra,
                           const double* __restrict__ rw, const double* __restrict__ rs,
                           const double* __restrict__ v, double* __restrict__ y)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= np) return;
    double s = 0.0;
    for (int q = 0; q < splits; ++q) s += part[q * np + j];
    for (int64_t p = cptr[j]; p < cptr[j + 1]; ++p) {
        const int64_t e = cent[p];
        if (!(flag[e] & bit)) continue;
        const double4 sv = src[crow[p]];
        const double4 vv = val[e];
        s += sv.x * vv.x + sv.y * vv.y + sv.z * vv.z + sv.w * vv.w;
    }
    if (kind[j] == BEM_DIELECTRIC) s += ra[j] * v[j];
    if (kind[j] == BEM_FLOATING) s += (0.5 * rw[j] + rs[j]) * v[np + aux[j]];
    y[j] = s;
}

// columns N+f: -sum of v over the rows of floating body f
__global__ void k_float_cols(int64_t np, const int32_t* __restrict__ rows, const int32_t* __restrict__ off,
                             const double* __restrict__ v, double* __restrict__ y)
{
    __shared__ double sh[256];
    const int f = blockIdx.x;
    double s = 0.0;
    for (int k = off[f] + threadIdx.x; k < off[f + 1]; k += blockDim.x) s += v[rows[k]];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) y[np + f] = -sh[0];
}

// ---------------------------------------------------------------- system gradient
// Row coefficients of -mu^T A u: kS_i on S_j(c_i), kG_i on G_j(c_i).
__device__ __forceinline__ void row_coef(int64_t i, int64_t np, const int32_t* kind, const int32_t* aux,
                                         const double* rb, const double* rw, const double* geo,
                                         const double* mu, double& kS, double* kG)
{
    const double* gp = geo + GEO_STRIDE * i;
    double c = 0.0;
    kS = 0.0;
    if (kind[i] == BEM_CONDUCTOR) {
        kS = -mu[i];
    } else if (kind[i] == BEM_FLOATING) {
        kS = -mu[i];
        c = -mu[np + aux[i]] * rw[i];
    } else {
        c = -mu[i] * rb[i];
    }
    kG[0] = c * gp[GEO_N]; kG[1] = c * gp[GEO_N + 1]; kG[2] = c * gp[GEO_N + 2];
}

// target side: t_i = sum_{j != i} u_j d(kS_i S_j + kG_i.G_j)/dx at c_i (partials per split)
template <bool F32, int Q>
__global__ void k_sys_rows(int64_t np, int g, const double* __restrict__ geo, const float4* __restrict__ hdr32,
                           const double4* __restrict__ hdr64, const float4* __restrict__ n32,
                           const double4* __restrict__ n64, const float4* __restrict__ t32,
                           const int32_t* __restrict__ kind, const int32_t* __restrict__ aux,
                           const double* __restrict__ rb, const double* __restrict__ rw,
                           const double* __restrict__ mu, const double* __restrict__ u,
                           int64_t per_split, double* __restrict__ part)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    const int64_t j0 = blockIdx.y * per_split, j1 = min(np, j0 + per_split);
    double kS, kG[3];
    row_coef(i, np, kind, aux, rb, rw, geo, mu, kS, kG);
    const double* gi = geo + GEO_STRIDE * i;
    const double x[3] = {gi[GEO_CTR], gi[GEO_CTR + 1], gi[GEO_CTR + 2]};
    const float4 tf = t32[i];
    double t[3] = {0.0, 0.0, 0.0};
    if (kS != 0.0 || kG[0] != 0.0 || kG[1] != 0.0 || kG[2] != 0.0) {
        for (int64_t j = j0; j < j1; ++j) {
            if (j == i) continue;
            const double* gp = geo + GEO_STRIDE * j;
            const bool far = F32 ? is_far32(tf.x, tf.y, tf.z, hdr32[j]) : is_far64(x[0], x[1], x[2], hdr64[j]);
            double F, d[3];
            if (far) {
                if (F32)
                    far_pair_grad<float, Q>(gp, n32, n64, j, g, x, kS, kG, true, false, F, d, nullptr);
                else
                    far_pair_grad<double, Q>(gp, n32, n64, j, g, x, kS, kG, true, false, F, d, nullptr);
            } else {
                near_pair_grad(gp, x, false, kS, kG, 0, F, d);
            }
            for (int c = 0; c < 3; ++c) t[c] += u[j] * d[c];
        }
    }
    double* o = part + (blockIdx.y * np + i) * 3;
    o[0] = t[0]; o[1] = t[1]; o[2] = t[2];
}

// source side: sum_{i != j} u_j d(kS_i S_j(c_i) + kG_i.G_j(c_i))/d(a_j,b_j,c_j)
template <bool F32, int Q>
__global__ void k_sys_cols(int64_t np, int g, const double* __restrict__ geo, const float4* __restrict__ hdr32,
                           const double4* __restrict__ hdr64, const float4* __restrict__ n32,
                           const double4* __restrict__ n64, const float4* __restrict__ t32,
                           const int32_t* __restrict__ kind, const int32_t* __restrict__ aux,
                           const double* __restrict__ rb, const double* __restrict__ rw,
                           const double* __restrict__ mu, const double* __restrict__ u,
                           int64_t per_split, double* __restrict__ part)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= np) return;
    const int64_t i0 = blockIdx.y * per_split, i1 = min(np, i0 + per_split);
    const double* gp = geo + GEO_STRIDE * j;
    double acc[9];
    for (int c = 0; c < 9; ++c) acc[c] = 0.0;
    for (int64_t i = i0; i < i1; ++i) {
        if (i == j) continue;
        double kS, kG[3];
        row_coef(i, np, kind, aux, rb, rw, geo, mu, kS, kG);
        if (kS == 0.0 && kG[0] == 0.0 && kG[1] == 0.0 && kG[2] == 0.0) continue;
        const double* gi = geo + GEO_STRIDE * i;
        const double x[3] = {gi[GEO_CTR], gi[GEO_CTR + 1], gi[GEO_CTR + 2]};
        const float4 tf = t32[i];
        const bool far = F32 ? is_far32(tf.x, tf.y, tf.z, hdr32[j]) : is_far64(x[0], x[1], x[2], hdr64[j]);
        double F, d[9];
        if (far) {
            if (F32)
                far_pair_grad<float, Q>(gp, n32, n64, j, g, x, kS, kG, false, true, F, nullptr, d);
            else
                far_pair_grad<double, Q>(gp, n32, n64, j, g, x, kS, kG, false, true, F, nullptr, d);
        } else {
            near_pair_grad(gp, x, false, kS, kG, 1, F, d);
        }
        for (int c = 0; c < 9; ++c) acc[c] += d[c];
    }
    double* o = part + (blockIdx.y * np + j) * 9;
    for (int c = 0; c < 9; ++c) o[c] = u[j] * acc[c];
}

// per row: the target-side sums mapped to the row triangle's corners (centroid),
// the own pair's total derivative, the normal and (neutrality rows) the area terms
__global__ void k_sys_row_terms(int64_t np, int splits_r, int splits_c, const double* __restrict__ geo,
                                const int32_t* __restrict__ kind, const int32_t* __restrict__ aux,
                                const double* __restrict__ rb, const double* __restrict__ rw,
                                const double* __restrict__ mu, const double* __restrict__ u,
                                const double* __restrict__ field, const double* __restrict__ Tf,
                                const double2* __restrict__ ceps, const double* __restrict__ area_f,
                                const double* __restrict__ part_r, const double* __restrict__ part_c,
                                double* __restrict__ gP)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= np) return;
    const double* gp = geo + GEO_STRIDE * i;
    double t[3] = {0.0, 0.0, 0.0}, out[9];
    for (int q = 0; q < splits_r; ++q)
        for (int c = 0; c < 3; ++c) t[c] += part_r[(q * np + i) * 3 + c];
    for (int c = 0; c < 9; ++c) out[c] = t[c % 3] / 3.0;  // centroid = mean of the corners
    for (int q = 0; q < splits_c; ++q)
        for (int c = 0; c < 9; ++c) out[c] += part_c[(q * np + i) * 9 + c];
    double kS, kG[3];
    row_coef(i, np, kind, aux, rb, rw, geo, mu, kS, kG);
    {   // own pair, total derivative (the centroid moves with the vertices)
        double F, d[9];
        near_pair_grad(gp, nullptr, true, kS, kG, 1, F, d);
        for (int c = 0; c < 9; ++c) out[c] += u[i] * d[c];
    }
    // normal: coefficient c n_i . E(c_i), d/dn = c E(c_i)
    double c = 0.0;
    if (kind[i] == BEM_FLOATING) c = -mu[np + aux[i]] * rw[i];
    if (kind[i] == BEM_DIELECTRIC) c = -mu[i] * rb[i];
    if (c != 0.0) {
        const double* E = field + 4 * i + 1;
        const double nx = gp[GEO_N], ny = gp[GEO_N + 1], nz = gp[GEO_N + 2];
        const double en = E[0] * nx + E[1] * ny + E[2] * nz;
        const double wn = 2.0 * gp[GEO_AREA];
        const double P[3] = {c * (E[0] - nx * en) / wn, c * (E[1] - ny * en) / wn, c * (E[2] - nz * en) / wn};
        const double e1[3] = {gp[3] - gp[0], gp[4] - gp[1], gp[5] - gp[2]};
        const double e2[3] = {gp[6] - gp[3], gp[7] - gp[4], gp[8] - gp[5]};
        const double e2P[3] = {e2[1] * P[2] - e2[2] * P[1], e2[2] * P[0] - e2[0] * P[2], e2[0] * P[1] - e2[1] * P[0]};
        const double Pe1[3] = {P[1] * e1[2] - P[2] * e1[1], P[2] * e1[0] - P[0] * e1[2], P[0] * e1[1] - P[1] * e1[0]};
        for (int q = 0; q < 3; ++q) {
            out[q] -= e2P[q];
            out[3 + q] += e2P[q] - Pe1[q];
            out[6 + q] += Pe1[q];
        }
    }
    if (kind[i] == BEM_FLOATING) {  // neutrality weights A_i / area_f of the summands tau_i
        const int f = aux[i];
        const double* E = field + 4 * i + 1;
        const double ti = 0.5 * u[i] + E[0] * gp[GEO_N] + E[1] * gp[GEO_N + 1] + E[2] * gp[GEO_N + 2];
        const double tau = ceps[i].x * ti + ceps[i].y * u[i];
        const double s = -mu[np + f] / area_f[f] * (tau - Tf[f]);
        double dA[9];
        area_grad(gp, dA);
        for (int q = 0; q < 9; ++q) out[q] += s * dA[q];
    }
    double* o = gP + 9 * i;
    for (int q = 0; q < 9; ++q) o[q] += out[q];
}

// neutrality means T_f = sum_{i in f} A_i tau_i / area_f, with the summand
// tau_i = ce_i (u_i/2 + (K'u)_i) + em_i u_i: ce = eps+ and em = 0 on a closed
// floating body, ce = eps+ - eps- and em = eps- on a sheet (Eq. sheets)
__global__ void k_float_means(int64_t np, const int32_t* __restrict__ rows, const int32_t* __restrict__ off,
                              const double* __restrict__ geo, const double* __restrict__ u,
                              const double* __restrict__ field, const double2* __restrict__ ceps,
                              const double* __restrict__ area_f, double* __restrict__ Tf)
{
    __shared__ double sh[256];
    const int f = blockIdx.x;
    double s = 0.0;
    for (int k = off[f] + threadIdx.x; k < off[f + 1]; k += blockDim.x) {
        const int i = rows[k];
        const double* gp = geo + GEO_STRIDE * i;
        const double* E = field + 4 * i + 1;
        const double ti = 0.5 * u[i] + E[0] * gp[GEO_N] + E[1] * gp[GEO_N + 1] + E[2] * gp[GEO_N + 2];
        s += gp[GEO_AREA] * (ceps[i].x * ti + ceps[i].y * u[i]);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) Tf[f] = sh[0] / area_f[f];
}

// V0 and eps gradients: one block per region
__global__ void k_region_grads(int64_t np, int nreg, const int32_t* __restrict__ region,
                               const int32_t* __restrict__ kind, const int32_t* __restrict__ aux,
                               const double* __restrict__ geo, const double* __restrict__ mu,
                               const double* __restrict__ u, const double* __restrict__ field,
                               const double* __restrict__ area_f, const int32_t* __restrict__ sheet,
                               double* __restrict__ gV0, double* __restrict__ geps)
{
    __shared__ double sh[3][256];
    const int r = blockIdx.x;
    double a = 0.0, bp = 0.0, bm = 0.0;
    for (int64_t i = threadIdx.x; i < np; i += blockDim.x) {
        if (region[i] != r) continue;
        const double* gp = geo + GEO_STRIDE * i;
        const double* E = field + 4 * i + 1;
        const double kp = E[0] * gp[GEO_N] + E[1] * gp[GEO_N + 1] + E[2] * gp[GEO_N + 2];
        if (kind[i] == BEM_CONDUCTOR) {
            a += mu[i];
        } else if (kind[i] == BEM_DIELECTRIC) {
            bp += -mu[i] * (0.5 * u[i] + kp);
            bm += -mu[i] * (0.5 * u[i] - kp);
        } else {  // floating body or sheet: the neutrality row's eps terms
            const double w = -mu[np + aux[i]] * gp[GEO_AREA] / area_f[aux[i]];
            bp += w * (0.5 * u[i] + kp);
            if (sheet[r]) bm += w * (0.5 * u[i] - kp);
        }
    }
    sh[0][threadIdx.x] = a; sh[1][threadIdx.x] = bp; sh[2][threadIdx.x] = bm;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
            for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (gV0) gV0[r] = sh[0][0];
        if (geps) { geps[2 * r] = sh[1][0]; geps[2 * r + 1] = sh[2][0]; }
    }
}

// corner gradients -> vertex gradients through the vertex -> (triangle, corner) lists
__global__ void k_gather_vertices(int64_t nv, const int64_t* __restrict__ vptr,
                                  const int64_t* __restrict__ vcorner, const double* __restrict__ gP,
                                  double* __restrict__ gX)
{
    const int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (v >= nv) return;
    double s[3] = {0.0, 0.0, 0.0};
    for (int64_t p = vptr[v]; p < vptr[v + 1]; ++p) {
        const int64_t jc = vcorner[p];  // 3 * triangle + corner
        for (int c = 0; c < 3; ++c) s[c] += gP[3 * jc + c];
    }
    gX[3 * v] = s[0]; gX[3 * v + 1] = s[1]; gX[3 * v + 2] = s[2];
}

}  // namespace

// ---------------------------------------------------------------- adjoint workspace
// Everything bem_adjoint needs, allocated once by bem_create (params.adjoint_lines > 0):
// checkpoints for `lines` lines at the default step limit, the step records of one
// segment of a backward batch, per-line gradient buffers (at most 64 MiB), and the
// buffers of the system gradient.
struct AdjWork {
    int64_t lines = 0;      // lines of one forward chunk at the default step limit
    int k = 128;            // checkpoint interval (steps)
    int64_t cp_cap = 0;     // checkpoints the store holds
    int64_t bw = 0;         // lines of one backward batch
    int splits = 1;         // target/source slices of the system-gradient kernels
    Ckpt* cp = nullptr;
    StepRec* tape = nullptr;
    int64_t *nrec = nullptr, *segn = nullptr;
    double *s0 = nullptr, *K = nullptr, *gul = nullptr, *gpl = nullptr, *lx = nullptr;
    int* sr = nullptr;
    int32_t* st = nullptr;
    double *gu = nullptr, *gPt = nullptr, *mu = nullptr, *gPs = nullptr, *af = nullptr, *Tf = nullptr;
    double *pr = nullptr, *pc = nullptr;
    double2* ceps = nullptr;
    int32_t* sheet = nullptr;
    int64_t *vptr = nullptr, *vc = nullptr;
};

// ---------------------------------------------------------------- transposed matvec
static int ensure_csc(bem_ctx* c)
{
    if (c->csc_ptr) return BEM_OK;
    const int64_t np = c->np, nnz = c->nnz;
    std::vector<int64_t> ptr(np + 1);
    std::vector<int32_t> col(nnz);
    BEM_CUDA_TRY(c, cudaMemcpy(ptr.data(), c->near_ptr, (np + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
    BEM_CUDA_TRY(c, cudaMemcpy(col.data(), c->near_col, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost));
    std::vector<int64_t> cptr(np + 1, 0), cent(nnz);
    std::vector<int32_t> crow(nnz);
    for (int64_t k = 0; k < nnz; ++k) cptr[col[k] + 1]++;
    for (int64_t j = 0; j < np; ++j) cptr[j + 1] += cptr[j];
    std::vector<int64_t> pos(cptr.begin(), cptr.end() - 1);
    for (int64_t i = 0; i < np; ++i)
        for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
            const int64_t p = pos[col[k]]++;
            crow[p] = (int32_t)i;
            cent[p] = k;
        }
    if (cudaMalloc((void**)&c->csc_ptr, (np + 1) * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc((void**)&c->csc_row, std::max<int64_t>(nnz, 1) * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc((void**)&c->csc_ent, std::max<int64_t>(nnz, 1) * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc((void**)&c->tsrc64, np * sizeof(double4)) != cudaSuccess ||
        cudaMalloc((void**)&c->tsrc32, np * sizeof(float4)) != cudaSuccess) {
        cudaGetLastError();
        return set_err(c, BEM_ERR_NOMEM, "adjoint workspace allocation failed");
    }
    BEM_CUDA_TRY(c, cudaMemcpy(c->csc_ptr, cptr.data(), (np + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    BEM_CUDA_TRY(c, cudaMemcpy(c->csc_row, crow.data(), nnz * sizeof(int32_t), cudaMemcpyHostToDevice));
    BEM_CUDA_TRY(c, cudaMemcpy(c->csc_ent, cent.data(), nnz * sizeof(int64_t), cudaMemcpyHostToDevice));
    return BEM_OK;
}

int matvecT_impl(bem_ctx* c, int precision, const double* v, double* y)
{
    if (!c->csc_ptr)
        return set_err(c, BEM_ERR_CAPACITY, "the transposed operator needs the adjoint workspace "
                       "(bem_create with params.adjoint_lines > 0)");
    const int64_t np = c->np;
    cudaStream_t s = c->stream;
    k_tsrc<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(np, c->row_kind, c->row_aux, c->row_b, c->row_w,
                                                        c->geo, v, c->tsrc64, c->tsrc32);
    BEM_LAUNCH_CHECK(c);
    const int64_t tiles = (np + 127) / 128;
    int splits = (int)std::max<int64_t>(1, std::min<int64_t>(64, (c->num_sms * 4) / std::max<int64_t>(tiles, 1)));
    if ((size_t)splits * np > c->part_cap) splits = (int)std::max<int64_t>(1, c->part_cap / np);
    const int64_t per = (np + splits - 1) / splits;
    dim3 grid((unsigned)tiles, (unsigned)splits);
    const bool f32 = precision == BEM_MIXED;
#define FT_CASE(G, QQ)                                                                              \
    case G:                                                                                         \
        if (f32)                                                                                    \
            k_far_T<true, QQ><<<grid, 128, 0, s>>>(np, c->tgt32, c->tgt64, c->hdr32, c->hdr64,      \
                                                   c->node32, c->node64, c->tsrc32, c->tsrc64, per, \
                                                   c->part);                                        \
        else                                                                                        \
            k_far_T<false, QQ><<<grid, 128, 0, s>>>(np, c->tgt32, c->tgt64, c->hdr32, c->hdr64,     \
                                                    c->node32, c->node64, c->tsrc32, c->tsrc64, per, \
                                                    c->part);                                       \
        break;
    switch (c->g) {
        FT_CASE(2, 4) FT_CASE(3, 9) FT_CASE(4, 16)
        default: return set_err(c, BEM_ERR_ARG, "far_order not compiled");
    }
#undef FT_CASE
    BEM_LAUNCH_CHECK(c);
    k_finish_T<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(
        np, splits, c->part, c->csc_ptr, c->csc_row, c->csc_ent, c->near_val, c->near_flag,
        (uint8_t)(f32 ? 1 : 2), c->tsrc64, c->row_kind, c->row_aux, c->row_a, c->row_w, c->row_s, v, y);
    BEM_LAUNCH_CHECK(c);
    if (c->nfloat > 0) {
        k_float_cols<<<c->nfloat, 256, 0, s>>>(np, c->float_rows, c->float_off, v, y);
        BEM_LAUNCH_CHECK(c);
    }
    return BEM_OK;
}

extern "C" int bem_matvec_transpose(bem_ctx* c, int32_t precision, const double* x, double* y)
{
    if (!c) return BEM_ERR_ARG;
    if (precision != BEM_FP64 && precision != BEM_MIXED)
        return set_err(c, BEM_ERR_ARG, "precision must be BEM_FP64 or BEM_MIXED");
    if (!x || !y) return set_err(c, BEM_ERR_ARG, "bem_matvec_transpose: NULL pointer");
    return matvecT_impl(c, precision, x, y);
}

// ---------------------------------------------------------------- bem_adjoint
template <class T>
static bool walloc(T** p, size_t n)
{
    if (cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    return true;
}

void adjoint_workspace_free(bem_ctx* c)
{
    AdjWork* W = c->adj;
    if (!W) return;
    void* ptrs[] = {W->cp, W->tape, W->nrec, W->segn, W->s0, W->K, W->gul, W->gpl, W->lx, W->sr, W->st,
                    W->gu, W->gPt, W->mu, W->gPs, W->af, W->Tf, W->pr, W->pc, W->ceps, W->sheet,
                    W->vptr, W->vc};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete W;
    c->adj = nullptr;
}

// bem_create: the adjoint workspace and the transposed operator's column lists
int adjoint_workspace_create(bem_ctx* c)
{
    if (c->prm.adjoint_lines <= 0) return BEM_OK;
    if (int rc = ensure_csc(c)) return rc;
    AdjWork* W = new AdjWork();
    c->adj = W;
    const int64_t np = c->np, nv = c->nv;
    W->k = std::max(1, (int)c->prm.adjoint_checkpoint);
    W->lines = c->prm.adjoint_lines;
    bem_trace_params tp;
    bem_default_trace_params(&tp);
    W->cp_cap = W->lines * ((tp.max_steps + W->k - 1) / W->k + 1);
    // backward batch: per-line gradient buffers (80 bytes per triangle) and one segment of
    // step records per line, each within 64 MiB
    W->bw = std::max<int64_t>(1, std::min<int64_t>(W->lines, ((int64_t)64 << 20) / (80 * np)));
    W->bw = std::max<int64_t>(1, std::min<int64_t>(W->bw, ((int64_t)64 << 20) / ((int64_t)W->k * sizeof(StepRec))));
    const int64_t tiles = (np + 127) / 128;
    W->splits = (int)std::max<int64_t>(1, std::min<int64_t>(64, (c->num_sms * 8) / std::max<int64_t>(tiles, 1)));
    const int64_t L = W->lines, nf = std::max(c->nfloat, 1);
    const int nreg = (int)c->regions.size();
    bool ok = walloc(&W->cp, W->cp_cap) && walloc(&W->tape, W->bw * W->k) && walloc(&W->nrec, L) &&
              walloc(&W->segn, W->bw) && walloc(&W->s0, L) && walloc(&W->K, L) &&
              walloc(&W->gul, W->bw * np) && walloc(&W->gpl, W->bw * 9 * np) && walloc(&W->lx, 3 * W->bw) &&
              walloc(&W->sr, L) && walloc(&W->st, L) && walloc(&W->gu, c->nunk) && walloc(&W->gPt, 9 * np) &&
              walloc(&W->mu, c->nunk) && walloc(&W->gPs, 9 * np) && walloc(&W->af, nf) && walloc(&W->Tf, nf) &&
              walloc(&W->pr, (size_t)W->splits * np * 3) && walloc(&W->pc, (size_t)W->splits * np * 9) &&
              walloc(&W->ceps, np) && walloc(&W->sheet, nreg) && walloc(&W->vptr, nv + 1) &&
              walloc(&W->vc, 3 * np);
    if (!ok) return set_err(c, BEM_ERR_NOMEM, "adjoint workspace allocation failed");
    cudaStream_t s = c->stream;
    // per row (ce, em) of the neutrality summand (see k_float_means), per region
    // whether it is a sheet, per floating body its area; vertex -> (triangle, corner) lists
    std::vector<double2> h_ceps(np, make_double2(0.0, 0.0));
    std::vector<double> h_af(nf, 0.0);
    std::vector<int32_t> h_sheet(nreg, 0);
    std::vector<double> g(GEO_STRIDE * np);
    std::vector<int32_t> tri(3 * np);
    BEM_CUDA_TRY(c, cudaMemcpyAsync(g.data(), c->geo, g.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(tri.data(), c->tri, 3 * np * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(c, cudaStreamSynchronize(s));
    for (int64_t i = 0; i < np; ++i) {
        const bem_region& R = c->regions[c->h_region[i]];
        if (R.kind == BEM_FLOATING || R.kind == BEM_SHEET) h_af[R.floating_id] += g[GEO_STRIDE * i + GEO_AREA];
        if (R.kind == BEM_FLOATING) h_ceps[i] = make_double2(R.eps_plus, 0.0);
        if (R.kind == BEM_SHEET) h_ceps[i] = make_double2(R.eps_plus - R.eps_minus, R.eps_minus);
    }
    for (int r = 0; r < nreg; ++r) h_sheet[r] = c->regions[r].kind == BEM_SHEET;
    std::vector<int64_t> vptr(nv + 1, 0), vc(3 * np);
    for (int64_t q = 0; q < 3 * np; ++q) vptr[tri[q] + 1]++;
    for (int64_t v = 0; v < nv; ++v) vptr[v + 1] += vptr[v];
    std::vector<int64_t> pos(vptr.begin(), vptr.end() - 1);
    for (int64_t q = 0; q < 3 * np; ++q) vc[pos[tri[q]]++] = q;
    BEM_CUDA_TRY(c, cudaMemcpyAsync(W->ceps, h_ceps.data(), np * sizeof(double2), cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(W->af, h_af.data(), nf * 8, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(W->sheet, h_sheet.data(), nreg * 4, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(W->vptr, vptr.data(), (nv + 1) * 8, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(W->vc, vc.data(), 3 * np * 8, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaStreamSynchronize(s));  // the host vectors end here
    return BEM_OK;
}

template <bool F32, int Q>
static int adjoint_run(bem_ctx* c, const TArgs& A, int64_t L, const double* seeds, const double* wts,
                       double* K_out, double* gX, double* gV0, double* geps, double tol)
{
    AdjWork& W = *c->adj;
    cudaStream_t s = c->stream;
    const int64_t np = c->np, nv = c->nv;
    const int precision = F32 ? BEM_MIXED : BEM_FP64;
    const int k = W.k;
    // checkpoints per line for this call's step limit, and the lines that fit
    const int64_t ncp = (A.max_steps + k - 1) / k + 1;
    const int64_t chunk = std::min<int64_t>(L, W.cp_cap / ncp);
    if (chunk < 1)
        return set_err(c, BEM_ERR_CAPACITY, "adjoint: max_steps %lld needs %lld checkpoints per line; the "
                       "workspace holds %lld", (long long)A.max_steps, (long long)ncp, (long long)W.cp_cap);
    constexpr size_t fsm = field_smem<F32, Q>();
    BEM_CUDA_TRY(c, allow_smem(k_adj_forward<F32, Q>, fsm));
    BEM_CUDA_TRY(c, allow_smem(k_adj_resume<F32, Q>, fsm));
    // one cluster size for the forward pass and every recomputed segment, so the
    // segments retrace the forward trajectories bit for bit
    const int ncl = tracer_cluster(np, chunk, c->num_sms, c->prm.trace_cluster);
    BEM_CUDA_TRY(c, cudaMemsetAsync(W.gu, 0, c->nunk * sizeof(double), s));
    BEM_CUDA_TRY(c, cudaMemsetAsync(W.gPt, 0, 9 * np * sizeof(double), s));
    std::vector<int64_t> h_n(chunk);
    std::vector<int32_t> h_st(chunk);
    for (int64_t c0 = 0; c0 < L; c0 += chunk) {
        const int64_t nc = std::min(chunk, L - c0);
        // 1. forward: K, status, step-record counts and a checkpoint every k steps
        const unsigned fgrid = lines_grid(k_adj_forward<F32, Q>, fsm, c->num_sms, nc, ncl);
        BEM_CUDA_TRY(c, cudaMemsetAsync(c->d_line_next, 0, sizeof(unsigned long long), s));
        BEM_CUDA_TRY(c, launch_lines(k_adj_forward<F32, Q>, fgrid, fsm, s, ncl, A, seeds + 3 * c0, nc,
                                     c->d_line_next, W.cp, ncp, k, W.nrec, W.s0, W.sr, W.K, W.st));
        BEM_LAUNCH_CHECK(c);
        if (K_out) BEM_CUDA_TRY(c, cudaMemcpyAsync(K_out + c0, W.K, nc * sizeof(double), cudaMemcpyDeviceToDevice, s));
        BEM_CUDA_TRY(c, cudaMemcpyAsync(h_n.data(), W.nrec, nc * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        BEM_CUDA_TRY(c, cudaMemcpyAsync(h_st.data(), W.st, nc * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        BEM_CUDA_TRY(c, cudaStreamSynchronize(s));
        for (int64_t l = 0; l < nc; ++l)
            if (h_st[l] == 2 || h_st[l] == -1)
                return set_err(c, BEM_ERR_ARG, "adjoint: line %lld ends with status %d (only r_max, step "
                               "limit and field floor are differentiated)", (long long)(c0 + l), h_st[l]);
        // 2. reverse sweep, a batch of lines at a time, segment by segment from the last:
        //    each segment is traced again from its checkpoint with a step record, then reversed
        for (int64_t b0 = 0; b0 < nc; b0 += W.bw) {
            const int64_t nb = std::min(W.bw, nc - b0);
            int64_t segs = 0;
            for (int64_t l = b0; l < b0 + nb; ++l) segs = std::max(segs, (h_n[l] + k - 1) / k);
            BEM_CUDA_TRY(c, cudaMemsetAsync(W.gul, 0, nb * np * sizeof(double), s));
            BEM_CUDA_TRY(c, cudaMemsetAsync(W.gpl, 0, nb * 9 * np * sizeof(double), s));
            BEM_CUDA_TRY(c, cudaMemsetAsync(W.lx, 0, 3 * nb * sizeof(double), s));
            const unsigned rgrid = lines_grid(k_adj_resume<F32, Q>, fsm, c->num_sms, nb, ncl);
            for (int64_t seg = segs - 1; seg >= 0; --seg) {
                BEM_CUDA_TRY(c, cudaMemsetAsync(c->d_line_next, 0, sizeof(unsigned long long), s));
                BEM_CUDA_TRY(c, launch_lines(k_adj_resume<F32, Q>, rgrid, fsm, s, ncl, A, nb, c->d_line_next,
                                             (const Ckpt*)(W.cp + b0 * ncp), ncp, k, seg,
                                             (const int64_t*)(W.nrec + b0), (const double*)(W.s0 + b0),
                                             (const int*)(W.sr + b0), W.tape, W.segn));
                BEM_LAUNCH_CHECK(c);
                k_adj_backward<F32, Q><<<(unsigned)nb, kT, 0, s>>>(A, c->g, W.tape, k, W.segn, W.s0 + b0,
                                                                   wts + c0 + b0, nb, W.gul, W.gpl, W.lx);
                BEM_LAUNCH_CHECK(c);
            }
            k_sum_lines<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(nb, np, W.gul, W.gu);
            BEM_LAUNCH_CHECK(c);
            k_sum_lines<<<(unsigned)((9 * np + 255) / 256), 256, 0, s>>>(nb, 9 * np, W.gpl, W.gPt);
            BEM_LAUNCH_CHECK(c);
        }
    }

    // 3. A^T mu = dJ/du
    int iters = 0;
    double rel = 0.0;
    int rc = solve_transpose(c, precision, W.gu, W.mu, tol, &iters, &rel);
    if (rc && rc != BEM_ERR_NOT_CONVERGED) return rc;

    // 4. -mu^T (dA/dX) u, V0 and eps gradients
    rc = matvec_impl(c, precision, 1, A.u, c->wvec, true);  // fills c->field with phi, E_PV at the centroids
    if (rc) return rc;
    const int nreg = (int)c->regions.size();
    if (c->nfloat > 0) {
        k_float_means<<<c->nfloat, 256, 0, s>>>(np, c->float_rows, c->float_off, c->geo, A.u, c->field, W.ceps,
                                                W.af, W.Tf);
        BEM_LAUNCH_CHECK(c);
    }
    const int64_t tiles = (np + 127) / 128;
    const int splits = W.splits;
    const int64_t per = (np + splits - 1) / splits;
    dim3 grid((unsigned)tiles, (unsigned)splits);
    k_sys_rows<F32, Q><<<grid, 128, 0, s>>>(np, c->g, c->geo, c->hdr32, c->hdr64, c->node32, c->node64,
                                            c->tgt32, c->row_kind, c->row_aux, c->row_b, c->row_w, W.mu, A.u,
                                            per, W.pr);
    BEM_LAUNCH_CHECK(c);
    k_sys_cols<F32, Q><<<grid, 128, 0, s>>>(np, c->g, c->geo, c->hdr32, c->hdr64, c->node32, c->node64,
                                            c->tgt32, c->row_kind, c->row_aux, c->row_b, c->row_w, W.mu, A.u,
                                            per, W.pc);
    BEM_LAUNCH_CHECK(c);
    BEM_CUDA_TRY(c, cudaMemcpyAsync(W.gPs, W.gPt, 9 * np * sizeof(double), cudaMemcpyDeviceToDevice, s));
    k_sys_row_terms<<<(unsigned)((np + 127) / 128), 128, 0, s>>>(
        np, splits, splits, c->geo, c->row_kind, c->row_aux, c->row_b, c->row_w, W.mu, A.u, c->field,
        W.Tf, W.ceps, W.af, W.pr, W.pc, W.gPs);
    BEM_LAUNCH_CHECK(c);
    k_region_grads<<<nreg, 256, 0, s>>>(np, nreg, c->d_region, c->row_kind, c->row_aux, c->geo, W.mu,
                                         A.u, c->field, W.af, W.sheet, gV0, geps);
    BEM_LAUNCH_CHECK(c);
    if (gX) {
        k_gather_vertices<<<(unsigned)((nv + 255) / 256), 256, 0, s>>>(nv, W.vptr, W.vc, W.gPs, gX);
        BEM_LAUNCH_CHECK(c);
    }
    BEM_CUDA_TRY(c, cudaStreamSynchronize(s));
    return BEM_OK;
}

extern "C" int bem_adjoint(bem_ctx* c, int32_t precision, const double* u, int64_t L, const double* seeds,
                           const bem_trace_params* tp, const double* dL_dK, double* K_out, double* gX,
                           double* gV0, double* geps)
{
    if (!c) return BEM_ERR_ARG;
    if (precision != BEM_FP64 && precision != BEM_MIXED)
        return set_err(c, BEM_ERR_ARG, "precision must be BEM_FP64 or BEM_MIXED");
    if (L < 1 || L > 0x7fffffff || !u || !seeds || !dL_dK)
        return set_err(c, BEM_ERR_ARG, "bem_adjoint: need L >= 1 and non-NULL u, seeds, dL_dK");
    if (!c->adj)
        return set_err(c, BEM_ERR_CAPACITY, "bem_adjoint needs the adjoint workspace (bem_create with "
                       "params.adjoint_lines > 0)");
    TArgs A;
    if (int rc = trace_args(c, tp, u, &A)) return rc;
    BEM_CUDA_TRY(c, cudaMemcpyToSymbolAsync(c_ru, c->h_rule_u.data(), c->g * sizeof(double), 0,
                                            cudaMemcpyHostToDevice, c->stream));
    BEM_CUDA_TRY(c, cudaMemcpyToSymbolAsync(c_rv, c->h_rule_v.data(), c->g * sizeof(double), 0,
                                            cudaMemcpyHostToDevice, c->stream));
    const double tol = precision == BEM_FP64 ? 1e-11 : 1e-6;
    const bool f32 = precision == BEM_MIXED;
    switch (c->g) {
#define AD_CASE(G, QQ)                                                                       \
    case G:                                                                                  \
        return f32 ? adjoint_run<true, QQ>(c, A, L, seeds, dL_dK, K_out, gX, gV0, geps, tol) \
                   : adjoint_run<false, QQ>(c, A, L, seeds, dL_dK, K_out, gX, gV0, geps, tol);
        AD_CASE(2, 4) AD_CASE(3, 9) AD_CASE(4, 16)
#undef AD_CASE
        default: return set_err(c, BEM_ERR_ARG, "bem_adjoint supports far_order 2..4");
    }
}

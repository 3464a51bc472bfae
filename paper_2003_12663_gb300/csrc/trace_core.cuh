// trace_core.cuh -- the field-line integrator shared by bem_trace_lines and the
// adjoint's recording forward pass (Sec. 1, Eq. Breakdowncrit), so that both
// compute the same trajectory bit for bit.
//
// One CTA traces one line.  Every field evaluation is a CTA-wide pass over all
// triangles: regular pairs by the Duffy/Gauss rule (FP32 or FP64), the others by the
// FP64 closed form, with the pair classification of the regular-pair kernels; the
// per-thread partial sums are added by a fixed-order block reduction whose result
// every thread receives.  The integrator (RK4 in arc length with K as extra state)
// then runs identically in all threads on those broadcast values, so control flow
// stays uniform and no thread ever waits on another beyond __syncthreads.
//
// Events (branch of alpha_eff at |E| = E0, |x| = r_max, entering another electrode)
// are located on the re-stepped RK4 step by the Illinois variant of regula falsi
// (at most 100 iterations); a step holds at most 4 events, the whole line at most
// max_steps steps, so every loop is bounded.
#pragma once

#include <cmath>

#include "bem_internal.cuh"

namespace tcore {

constexpr int kT = 256;
constexpr int kWarps = kT / 32;

struct TArgs {
    int64_t np;
    const float4* hdr32;
    const double4* hdr64;
    const float4* node32;
    const double4* node64;
    const double* geo;
    const double* u;
    const int32_t* region;
    const int32_t* electrode;
    double h, r_max, c, E0, d, e_floor;
    int64_t max_steps;
    const float4* nrm32;  // [np] FP32 normal, region index in the bits of w
};

// The FP32 field evaluation streams the triangles through shared memory in chunks
// of TC (nodes, classification header, normal + region, density), double-buffered
// with asynchronous copies so the loads of chunk c+1 overlap the work on chunk c.
// Thread t takes triangle c*TC + t of every chunk: with TC = kT that is the
// triangle sequence t, t + kT, t + 2 kT, ... of a plain strided loop.
template <int Q>
struct Stage32 {
    static constexpr int TC = Q <= 16 ? kT : kT / 2;  // larger rules: half chunks fit the 227 KB
    float4 node[2][TC * Q];
    float4 hdr[2][TC];
    float4 nrm[2][TC];
    double u[2][TC];
};

// dynamic shared memory a kernel running trace_line<F32, Q> must be launched with
template <bool F32, int Q>
constexpr size_t field_smem()
{
    return F32 ? sizeof(Stage32<Q>) : 0;
}

// allow a kernel more than the default 48 KB of dynamic shared memory
template <class Kernel>
inline cudaError_t allow_smem(Kernel k, size_t bytes)
{
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

__device__ __forceinline__ void cp_async16(void* s, const void* g)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(g) : "memory");
}

__device__ __forceinline__ void cp_async8(void* s, const void* g)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(g) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// issue the copies of triangles [c0, c0 + n) into buffer b
template <int Q>
__device__ __forceinline__ void stage_chunk(const TArgs& A, Stage32<Q>& S, int b, int64_t c0, int n)
{
    const float4* gn = A.node32 + c0 * Q;
    for (int k = threadIdx.x; k < n * Q; k += kT) cp_async16(&S.node[b][k], gn + k);
    for (int k = threadIdx.x; k < n; k += kT) {
        cp_async16(&S.hdr[b][k], A.hdr32 + c0 + k);
        cp_async16(&S.nrm[b][k], A.nrm32 + c0 + k);
        cp_async8(&S.u[b][k], A.u + c0 + k);
    }
}

struct V4 {
    double x, y, z, w;  // field (x,y,z) and the electrode indicator (w)
};

__device__ __forceinline__ double wsum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum over the CTA in a fixed order; every thread gets the same result
__device__ inline V4 block_sum(V4 v, double* sh)
{
    v.x = wsum(v.x); v.y = wsum(v.y); v.z = wsum(v.z); v.w = wsum(v.w);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) {
        sh[warp] = v.x; sh[kWarps + warp] = v.y; sh[2 * kWarps + warp] = v.z; sh[3 * kWarps + warp] = v.w;
    }
    __syncthreads();
    V4 r = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        r.x += sh[w]; r.y += sh[kWarps + w]; r.z += sh[2 * kWarps + w]; r.w += sh[3 * kWarps + w];
    }
    return r;
}

// E(x) and the indicator sum_{j in other electrodes} G_j(x).n_j
template <bool F32, int Q>
__device__ __noinline__ V4 cta_field(const TArgs& A, const double* x, int seed_region, double* sh)
{
    const float xf = __double2float_rn(x[0]), yf = __double2float_rn(x[1]), zf = __double2float_rn(x[2]);
    float fx = 0.f, fy = 0.f, fz = 0.f, fi = 0.f;      // FP32 regular pairs (times 4 pi)
    double qx = 0.0, qy = 0.0, qz = 0.0, qi = 0.0;     // FP64 regular pairs (times 4 pi)
    double nx_ = 0.0, ny_ = 0.0, nz_ = 0.0, ni = 0.0;  // closed-form pairs
    // a near pair: the closed form in FP64
    auto near_pair = [&](int64_t j, double uj, bool mark) {
        const double* gp = A.geo + GEO_STRIDE * j;
        double S, Gx, Gy, Gz;
        tri_closed_form(gp, x[0], x[1], x[2], false, S, Gx, Gy, Gz);
        nx_ = fma(uj, Gx, nx_); ny_ = fma(uj, Gy, ny_); nz_ = fma(uj, Gz, nz_);
        if (mark) ni += Gx * gp[GEO_N] + Gy * gp[GEO_N + 1] + Gz * gp[GEO_N + 2];
    };
    if constexpr (F32) {
        extern __shared__ __align__(16) unsigned char tcore_dyn[];
        Stage32<Q>& S = *reinterpret_cast<Stage32<Q>*>(tcore_dyn);
        constexpr int TC = Stage32<Q>::TC;
        const int64_t nch = (A.np + TC - 1) / TC;
        const int t = threadIdx.x;
        stage_chunk<Q>(A, S, 0, 0, (int)min((int64_t)TC, A.np));
        cp_async_commit();
        for (int64_t c = 0; c < nch; ++c) {
            const int b = (int)(c & 1);
            if (c + 1 < nch) {
                const int64_t c1 = (c + 1) * TC;
                stage_chunk<Q>(A, S, b ^ 1, c1, (int)min((int64_t)TC, A.np - c1));
                cp_async_commit();
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            const int64_t j = c * TC + t;
            if (t < TC && j < A.np) {
                const float4 nv = S.nrm[b][t];
                const int rj = __float_as_int(nv.w);
                const bool mark = rj != seed_region && A.electrode[rj] != 0;
                const double uj = S.u[b][t];
                if (is_far32(xf, yf, zf, S.hdr[b][t])) {
                    float gx = 0.f, gy = 0.f, gz = 0.f;
#pragma unroll
                    for (int k = 0; k < Q; ++k) {
                        const float4 nd = S.node[b][t * Q + k];
                        const float dx = xf - nd.x, dy = yf - nd.y, dz = zf - nd.z;
                        const float ri = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, 1e-20f))));
                        const float t3 = nd.w * ri * ri * ri;
                        gx = fmaf(t3, dx, gx); gy = fmaf(t3, dy, gy); gz = fmaf(t3, dz, gz);
                    }
                    const float uf = __double2float_rn(uj);
                    fx = fmaf(uf, gx, fx); fy = fmaf(uf, gy, fy); fz = fmaf(uf, gz, fz);
                    if (mark) fi += gx * nv.x + gy * nv.y + gz * nv.z;
                } else {
                    near_pair(j, uj, mark);
                }
            }
            __syncthreads();  // buffer b is refilled in the next iteration
        }
    } else {
        for (int64_t j = threadIdx.x; j < A.np; j += kT) {
            const int rj = A.region[j];
            const bool mark = rj != seed_region && A.electrode[rj] != 0;
            const double uj = A.u[j];
            if (is_far64(x[0], x[1], x[2], A.hdr64[j])) {
                const double* gp = A.geo + GEO_STRIDE * j;
                double gx = 0.0, gy = 0.0, gz = 0.0;
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    const double4 nd = A.node64[j * Q + k];
                    const double dx = x[0] - nd.x, dy = x[1] - nd.y, dz = x[2] - nd.z;
                    const double ri = rsqrt(fma(dx, dx, fma(dy, dy, fma(dz, dz, 1e-200))));
                    const double t3 = nd.w * ri * ri * ri;
                    gx = fma(t3, dx, gx); gy = fma(t3, dy, gy); gz = fma(t3, dz, gz);
                }
                qx = fma(uj, gx, qx); qy = fma(uj, gy, qy); qz = fma(uj, gz, qz);
                if (mark) qi += gx * gp[GEO_N] + gy * gp[GEO_N + 1] + gz * gp[GEO_N + 2];
            } else {
                near_pair(j, uj, mark);
            }
        }
    }
    V4 v;
    v.x = nx_ + kInv4Pi * (qx + (double)fx);
    v.y = ny_ + kInv4Pi * (qy + (double)fy);
    v.z = nz_ + kInv4Pi * (qz + (double)fz);
    v.w = ni + kInv4Pi * (qi + (double)fi);
    return block_sum(v, sh);
}

__device__ __forceinline__ double norm3(double a, double b, double c) { return sqrt(a * a + b * b + c * c); }

__device__ __forceinline__ double alpha_eff(const TArgs& A, double Em, int side)
{
    return side > 0 ? A.c * (Em - A.E0) * (Em - A.E0) : -A.d;
}

// one RK4 step of length s from (x, K); E0c: field at x if known
template <bool F32, int Q>
__device__ void rk4(const TArgs& A, int seed_region, double s0, int side, const double* x, double K,
                    double s, const V4* E0c, double* x1, double& K1, double* sh)
{
    double k[4][3], a[4], y[3] = {x[0], x[1], x[2]};
    for (int st = 0; st < 4; ++st) {
        const V4 E = (st == 0 && E0c) ? *E0c : cta_field<F32, Q>(A, y, seed_region, sh);
        const double Em = norm3(E.x, E.y, E.z);
        k[st][0] = E.x * (s0 / Em);
        k[st][1] = E.y * (s0 / Em);
        k[st][2] = E.z * (s0 / Em);
        a[st] = alpha_eff(A, Em, side);
        if (st < 3) {
            const double f = st < 2 ? 0.5 * s : s;
            for (int c = 0; c < 3; ++c) y[c] = x[c] + k[st][c] * f;
        }
    }
    for (int c = 0; c < 3; ++c)
        x1[c] = x[c] + ((k[0][c] + (k[1][c] + k[2][c]) * 2.0) + k[3][c]) * (s / 6.0);
    K1 = K + s / 6.0 * (a[0] + 2.0 * (a[1] + a[2]) + a[3]);
}

enum { EV_ALPHA = 0, EV_RMAX = 1, EV_ELECTRODE = 2 };

template <bool F32, int Q>
__device__ double event_g(const TArgs& A, int seed_region, double s0, int side, const double* x,
                          double K, const V4* E0c, double sig, int ev, double* sh)
{
    double x1[3], K1;
    rk4<F32, Q>(A, seed_region, s0, side, x, K, sig, E0c, x1, K1, sh);
    if (ev == EV_RMAX) return norm3(x1[0], x1[1], x1[2]) - A.r_max;
    const V4 E = cta_field<F32, Q>(A, x1, seed_region, sh);
    if (ev == EV_ALPHA) return norm3(E.x, E.y, E.z) - A.E0;
    return E.w + 0.5;
}

template <bool F32, int Q>
__device__ double illinois(const TArgs& A, int seed_region, double s0, int side, const double* x,
                           double K, const V4* E0c, double b, double ga, double gb, int ev, double* sh)
{
    double a = 0.0, c = b;
    int last = 0;
    for (int it = 0; it < 100; ++it) {
        c = (ga * b - gb * a) / (ga - gb);
        const double gc = event_g<F32, Q>(A, seed_region, s0, side, x, K, E0c, c, ev, sh);
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
        if (b - a <= 1e-14 * A.h) break;
    }
    return c;
}

// Sub-step kinds reported to a recorder.
enum { SUB_PLAIN = 0, SUB_ALPHA = 1, SUB_RMAX = 2, SUB_ELECTRODE = 3 };

// A recorder that records nothing (bem_trace_lines).
struct NoRec {
    __device__ void begin(double s0, int seed_region) {}
    __device__ void step(int64_t step, const double* x, double K, int side) {}
    __device__ void sub(int64_t step, int k, double sig, int kind) {}
};

// Trace one line from seed xs; all threads of the CTA call this with the same
// arguments.  Outputs (K, status, steps, end point) are returned to every thread.
template <bool F32, int Q, class Rec>
__device__ void trace_line(const TArgs& A, const double* xs, Rec& rec, double& K_out, int& st_out,
                           int64_t& ns_out, double* xe_out, double* sh, double* s_bd, long long* s_bj)
{
    double x[3] = {xs[0], xs[1], xs[2]};
    double K = 0.0;
    // electrode of the seed: the triangle with the nearest centroid (first on ties)
    double bd = 1e300;
    long long bj = 0;
    for (int64_t j = threadIdx.x; j < A.np; j += kT) {
        const double* c = A.geo + GEO_STRIDE * j + GEO_CTR;
        const double dd = (x[0] - c[0]) * (x[0] - c[0]) + (x[1] - c[1]) * (x[1] - c[1]) + (x[2] - c[2]) * (x[2] - c[2]);
        if (dd < bd) { bd = dd; bj = j; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double od = __shfl_xor_sync(0xffffffffu, bd, o);
        const long long oj = __shfl_xor_sync(0xffffffffu, bj, o);
        if (od < bd || (od == bd && oj < bj)) { bd = od; bj = oj; }
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) { s_bd[threadIdx.x >> 5] = bd; s_bj[threadIdx.x >> 5] = bj; }
    __syncthreads();
    bd = s_bd[0]; bj = s_bj[0];
    for (int w = 1; w < kWarps; ++w)
        if (s_bd[w] < bd || (s_bd[w] == bd && s_bj[w] < bj)) { bd = s_bd[w]; bj = s_bj[w]; }
    const int seed_region = A.region[bj];
    const double* nb = A.geo + GEO_STRIDE * bj + GEO_N;
    V4 E = cta_field<F32, Q>(A, x, -2, sh);
    const double s0 = (E.x * nb[0] + E.y * nb[1] + E.z * nb[2]) >= 0.0 ? 1.0 : -1.0;
    int side = norm3(E.x, E.y, E.z) > A.E0 ? 1 : -1;
    rec.begin(s0, seed_region);
    int st = 3;
    int64_t step = 0;
    bool have = false;  // E holds the field at x (with the seed's indicator)
    for (; step < A.max_steps; ++step) {
        if (!have) E = cta_field<F32, Q>(A, x, seed_region, sh);
        have = false;
        const double Em = norm3(E.x, E.y, E.z);
        if (!isfinite(Em)) { st = -1; break; }
        if (Em < A.e_floor) { st = 4; break; }
        rec.step(step, x, K, side);
        double rem = A.h;
        bool done = false, first = true;
        for (int nev = 0; rem > 0.0 && nev < 4; ++nev) {
            const V4* Ec = first ? &E : nullptr;
            double x1[3], K1;
            rk4<F32, Q>(A, seed_region, s0, side, x, K, rem, Ec, x1, K1, sh);
            const V4 E1 = cta_field<F32, Q>(A, x1, seed_region, sh);
            const double E1m = norm3(E1.x, E1.y, E1.z);
            double best = 2.0 * rem;
            int which = -1;
            if ((E1m > A.E0) != (side > 0)) {
                const double ga = event_g<F32, Q>(A, seed_region, s0, side, x, K, Ec, 0.0, EV_ALPHA, sh);
                const double sg = illinois<F32, Q>(A, seed_region, s0, side, x, K, Ec, rem, ga, E1m - A.E0, EV_ALPHA, sh);
                if (sg < best) { best = sg; which = EV_ALPHA; }
            }
            const double r1 = norm3(x1[0], x1[1], x1[2]);
            if (r1 >= A.r_max) {
                const double sg = illinois<F32, Q>(A, seed_region, s0, side, x, K, Ec, rem,
                                                   norm3(x[0], x[1], x[2]) - A.r_max, r1 - A.r_max, EV_RMAX, sh);
                if (sg < best) { best = sg; which = EV_RMAX; }
            }
            if (E1.w < -0.5) {
                const double ga = event_g<F32, Q>(A, seed_region, s0, side, x, K, Ec, 0.0, EV_ELECTRODE, sh);
                const double sg = illinois<F32, Q>(A, seed_region, s0, side, x, K, Ec, rem, ga, E1.w + 0.5, EV_ELECTRODE, sh);
                if (sg < best) { best = sg; which = EV_ELECTRODE; }
            }
            if (which < 0) {
                rec.sub(step, nev, rem, SUB_PLAIN);
                x[0] = x1[0]; x[1] = x1[1]; x[2] = x1[2];
                K = K1;
                E = E1;
                have = true;
                rem = 0.0;
                break;
            }
            rec.sub(step, nev, best, which == EV_ALPHA ? SUB_ALPHA : (which == EV_RMAX ? SUB_RMAX : SUB_ELECTRODE));
            double xn[3], Kn;
            rk4<F32, Q>(A, seed_region, s0, side, x, K, best, Ec, xn, Kn, sh);
            x[0] = xn[0]; x[1] = xn[1]; x[2] = xn[2];
            K = Kn;
            first = false;
            if (which == EV_ALPHA) {
                side = -side;
                rem -= best;
                continue;
            }
            st = which == EV_RMAX ? 1 : 2;
            done = true;
            break;
        }
        if (done) break;
    }
    K_out = K;
    st_out = st;
    ns_out = step;
    xe_out[0] = x[0]; xe_out[1] = x[1]; xe_out[2] = x[2];
}

}  // namespace tcore

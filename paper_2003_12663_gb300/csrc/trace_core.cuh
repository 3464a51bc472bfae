// trace_core.cuh -- the field-line integrator shared by bem_trace_lines,
// bem_batch_trace and the adjoint's recording forward pass (Sec. 1, Eq.
// Breakdowncrit), so that all of them compute the same trajectory bit for bit.
//
// A tracer CTA of kLW warps traces up to kLW lines at a time, one per warp.  Each
// warp runs the integrator of its own line (RK4 in arc length with K as extra
// state, FP64, identical in all 32 lanes so control flow is warp-uniform).  Field
// evaluations are collective rounds: every warp posts the point it needs (or
// nothing), then all threads evaluate the field at all posted points in one pass
// over the triangles -- each staged quadrature node serves every posted target --
// and each warp takes its own result.  Regular pairs by the Duffy/Gauss rule (FP32
// or FP64), the other pairs by the FP64 closed form, with the pair classification of
// the regular-pair kernels.  A target's sums depend on its own point only: thread t
// always takes the same triangles in the same order and every reduction runs per
// target, so a line's result does not depend on which lines share its rounds.
//
// Events (branch of alpha_eff at |E| = E0, |x| = r_max, entering another electrode)
// are located on the re-stepped RK4 step by the Illinois variant of regula falsi
// (at most 100 iterations); a step holds at most 4 events, the whole line at most
// max_steps steps, so every loop is bounded.  Warps synchronise through CTA
// barriers that every warp reaches once per round (a warp without a line joins
// the rounds until no warp has one).  On meshes of kSplitMin triangles or more a
// launch may be made of clusters of up to kCl CTAs: the leader runs the lines, each
// helper sweeps its own part of the triangles (every ncl-th group of 32, so that the
// near pairs of a point spread over the cluster) in every round of its leader, and all
// meet at the hardware cluster barrier twice per round (the round's points pushed
// into the helpers' shared memory; then the leader reads each helper's partial sums
// from the helper's shared memory, in rank order).  Every CTA of a cluster runs the
// same fixed sequence of barriers, paired one to one, and no CTA waits on a CTA
// outside its own cluster.  The sums are grouped by the cluster's parts, so on such
// meshes launches of different cluster sizes agree to rounding, not bit for bit.
#pragma once

#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "bem_internal.cuh"

namespace tcore {

namespace cg = cooperative_groups;

constexpr int kT = 256;          // threads of the adjoint's CTA-wide passes
constexpr int kWarps = kT / 32;
constexpr int kLW = 8;           // lines in flight per tracer CTA, one per warp
constexpr int kLT = 32 * kLW;    // threads per tracer CTA
constexpr int kCl = 8;           // largest tracer cluster (the portable limit)
constexpr int64_t kSplitMin = 8192;  // meshes of this many triangles or more may be split over a cluster
constexpr int64_t kPartMin = 2048;   // an automatic split leaves every CTA at least this many triangles

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
    const float* u32;     // [np] u rounded to FP32 (the regular pairs' density)
};


struct V4 {
    double x, y, z, w;  // field (x,y,z) and the electrode indicator (w)
};

__device__ __forceinline__ double wsum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ float wsumf(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// barrier of the kLT threads of a tracer CTA (its own id: warps reach it from
// different places of the integrator)
__device__ __forceinline__ void cta_bar() { asm volatile("bar.sync 1, %0;\n" ::"n"(kLT) : "memory"); }

constexpr int kNearCap = 32;     // near pairs a (warp, target) list holds before it is evaluated

// One round's requests and per-warp partial sums, in shared memory.
struct Round {
    double x[kLW][3];     // point posted by warp w
    int sr[kLW];          // its seed region (triangles of other electrodes feed the indicator)
    int act[kLW];         // 1 if warp w posted a point
    float F[kLW][kLW][4];   // [target][warp] FP32 regular pairs (times 4 pi)
    double N[kLW][kLW][4];  // [target][warp] closed-form pairs
    double G[kLW][kLW][4];  // [target][warp] FP64 regular pairs (times 4 pi)
    int32_t near[kLW][kLW][kNearCap];  // [warp][target slot] triangles of near pairs found
    // cluster exchange: the leader pushes x, sr, act, args and exit into each helper's
    // round; a helper leaves its part of the field at each posted point in P (sums over
    // its warps in order: FP32 regular, closed-form, FP64 regular pairs, 4 components
    // each), which the leader reads after the round's second cluster barrier
    TArgs args;
    int exit;
    double P[kLW][12];
};

// the triangles [j0, j1) that the cluster's CTA of this rank sweeps in every round of
// the FP64 form: a mesh of kSplitMin triangles or more is split into ncl parts of
// whole 256-triangle chunks; a smaller mesh is swept by the leader alone, so its sums
// do not depend on the cluster size
__device__ __forceinline__ void rank_range(int64_t np, int rank, int ncl, int64_t& j0, int64_t& j1)
{
    const int parts = np >= kSplitMin ? ncl : 1;
    const int64_t per = ((np + parts - 1) / parts + 255) / 256 * 256;
    j0 = min(np, (int64_t)rank * per);
    j1 = min(np, j0 + per);
}

// The FP32 form deals the mesh's 32-triangle groups to the cluster's CTAs in turn:
// group g goes to rank g mod parts (parts = ncl on a mesh of kSplitMin triangles or
// more, else 1: the leader alone).  Neighbouring triangles, and with them the near
// pairs of a point (FP64 closed form, the slow part of a round near the surfaces),
// land on different CTAs, so no CTA keeps the others waiting at the cluster barrier
// with all of them.  Chunk c of the rank holds its groups c*GW .. c*GW+GW-1 (GW
// groups per chunk, one per warp); every group starts on a multiple of 32 triangles,
// so the staging copies stay aligned.
struct RankGroups {
    int rank = 0, parts = 1;
    int64_t ngroups = 0;  // groups of this rank
    __device__ RankGroups(int64_t np, int r, int ncl)
    {
        parts = np >= kSplitMin ? ncl : 1;
        rank = r;
        const int64_t G = (np + 31) / 32;
        ngroups = (r < parts && r < G) ? (G - 1 - r) / parts + 1 : 0;
    }
    // first triangle of the rank's k-th group, or -1 past its last
    __device__ __forceinline__ int64_t first(int64_t k) const
    {
        return k < ngroups ? (k * parts + rank) * 32 : -1;
    }
};

// cluster size of a tracer launch over meshes of at most np triangles and `lines`
// lines, on a GPU of num_sms SMs (one tracer CTA per SM): `want` (1..kCl) if given;
// else the largest size that still leaves every CTA kPartMin triangles and whose
// clusters, a GPU full of them with kLW lines each, hold at least a quarter of the
// lines at once -- few lines get wide clusters (the rounds of a lone line, and the
// tail of every run, are swept by several SMs), many lines plain CTAs (no exchange;
// every SM is already busy with lines)
inline int tracer_cluster(int64_t np, int64_t lines, int num_sms, int want = 0)
{
    if (want > 0) return std::min(want, kCl);
    if (np < kSplitMin) return 1;
    int ncl = 1;
    for (int c = 2; c <= kCl; ++c) {
        if (np / c < kPartMin) break;
        const int64_t clusters = std::max(1, num_sms / c);
        if (lines > 4 * clusters * kLW) break;
        ncl = c;
    }
    return ncl;
}

// The FP32 evaluation streams the triangles through shared memory in chunks of TC
// (nodes, classification header, normal + region, density) with an NS-stage ring of
// asynchronous copies: while chunk c is evaluated the copies of chunks c+1 .. c+NS-1
// are in flight, so a round with a single posted point is not left waiting on L2.
template <int Q>
struct Stage32 {
    static constexpr int TC = Q <= 16 ? kLT : kLT / 2;  // larger rules: half chunks
    static constexpr int NS = Q <= 9 ? 4 : 2;           // stages (184 KB for Q = 9)
    float4 node[NS][TC * Q];
    float4 hdr[NS][TC];
    float4 nrm[NS][TC];
    float u[NS][TC];
};

// dynamic shared memory a tracer kernel for (F32, Q) must be launched with
template <bool F32, int Q>
constexpr size_t field_smem()
{
    return F32 ? sizeof(Stage32<Q>) : 0;
}

// let a kernel take `bytes` of dynamic shared memory on top of its static shared
// memory (past 48 KB in total the kernel must opt in)
template <class Kernel>
inline cudaError_t allow_smem(Kernel k, size_t bytes)
{
    if (bytes == 0) return cudaSuccess;
    return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

__device__ __forceinline__ void cp_async16(void* s, const void* g)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(g) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// issue the copies of the calling warp's triangles of the rank's chunk c into buffer
// b: warp w evaluates group c*GW + w of the rank (lane i its triangle i), and copies
// exactly those 32 triangles (coalesced) into slots w*32 .. w*32+31.
// The ring is thus private to each warp: a warp waits for its own copies and
// synchronises with its own lanes, never with the other warps of the CTA.
template <int Q>
__device__ __forceinline__ void stage_chunk(const TArgs& A, Stage32<Q>& S, int b, const RankGroups& RG, int64_t c)
{
    constexpr int GW = Stage32<Q>::TC / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (w >= GW) return;
    const int64_t j0 = RG.first(c * GW + w);  // this warp's group
    if (j0 < 0) return;
    const int nk = (int)min((int64_t)32, A.np - j0);
    const int k0 = w * 32;
    const float4* gn = A.node32 + j0 * Q;
    float4* sn = &S.node[b][k0 * Q];
    for (int k = lane; k < nk * Q; k += 32) cp_async16(sn + k, gn + k);
    if (lane < nk) {
        cp_async16(&S.hdr[b][k0 + lane], A.hdr32 + j0 + lane);
        cp_async16(&S.nrm[b][k0 + lane], A.nrm32 + j0 + lane);
    }
    // u: 16-byte copies of four values (j0 is a multiple of 32), plain loads for the rest
    const int n4 = nk / 4;
    if (lane < n4) cp_async16(&S.u[b][k0 + 4 * lane], A.u32 + j0 + 4 * lane);
    if (4 * n4 + lane < nk) S.u[b][k0 + 4 * n4 + lane] = A.u32[j0 + 4 * n4 + lane];
}

// The field at the posted points (slots 0..nt-1: the posting warps in order; NT is
// nt rounded up to a power of two, the extra slots repeat the last point and are not
// stored): E(x) and the indicator sum_{j in other electrodes} G_j(x).n_j, as
// per-warp partial sums in R (all threads call this).
//  * FP32 form: regular pairs from the staged chunks, every node applied to all NT
//    slots (independent chains, no branch between slots).  Near pairs are only
//    listed during the sweep -- per warp and per slot, in the order found -- and
//    evaluated 32 at a time with the FP64 closed form by all lanes of the warp, so
//    the slow FP64 units are busy with full warps instead of one lane at a time;
//    each batch is summed over the warp and added to R.N by lane 0.
//  * FP64 form: one plain strided pass per slot, FP64 regular pairs, closed form in
//    place.
template <bool F32, int Q, int NT>
__device__ void eval_targets(const TArgs& A, Round& R, unsigned amask, int nt, int rank, int ncl)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int tk[NT];
#pragma unroll
    for (int s = 0; s < NT; ++s) tk[s] = (int)__fns(amask, 0, min(s, nt - 1) + 1);
    if (lane == 0)
#pragma unroll
        for (int s = 0; s < NT; ++s)
            if (s < nt)
#pragma unroll
                for (int c = 0; c < 4; ++c) R.N[tk[s]][warp][c] = 0.0;
    __syncwarp();
    // the closed form of near pair (slot s, triangle j); the contribution to E and to
    // the indicator is added to d[0..3]
    auto near_pair = [&](int s, int64_t j, double* d) {
        const double* gp = A.geo + GEO_STRIDE * j;
        const int rj = A.region[j];
        const bool mark = A.electrode[rj] != 0 && rj != R.sr[tk[s]];
        const double uj = A.u[j];
        double S, Gx, Gy, Gz;
        tri_closed_form(gp, R.x[tk[s]][0], R.x[tk[s]][1], R.x[tk[s]][2], false, S, Gx, Gy, Gz);
        d[0] = fma(uj, Gx, d[0]); d[1] = fma(uj, Gy, d[1]); d[2] = fma(uj, Gz, d[2]);
        if (mark) d[3] += Gx * gp[GEO_N] + Gy * gp[GEO_N + 1] + Gz * gp[GEO_N + 2];
    };
    if constexpr (F32) {
        float xf[NT], yf[NT], zf[NT];
        int sr[NT];
        float fx[NT], fy[NT], fz[NT], fi[NT];  // FP32 regular pairs (times 4 pi)
#pragma unroll
        for (int s = 0; s < NT; ++s) {
            sr[s] = R.sr[tk[s]];
            xf[s] = __double2float_rn(R.x[tk[s]][0]);
            yf[s] = __double2float_rn(R.x[tk[s]][1]);
            zf[s] = __double2float_rn(R.x[tk[s]][2]);
            fx[s] = fy[s] = fz[s] = fi[s] = 0.f;
        }
        float2 x2[NT / 2 > 0 ? NT / 2 : 1], y2[NT / 2 > 0 ? NT / 2 : 1], z2[NT / 2 > 0 ? NT / 2 : 1];
#pragma unroll
        for (int s = 0; s < NT / 2; ++s) {
            x2[s] = make_float2(xf[2 * s], xf[2 * s + 1]);
            y2[s] = make_float2(yf[2 * s], yf[2 * s + 1]);
            z2[s] = make_float2(zf[2 * s], zf[2 * s + 1]);
        }
        extern __shared__ __align__(16) unsigned char tcore_dyn[];
        Stage32<Q>& S = *reinterpret_cast<Stage32<Q>*>(tcore_dyn);
        constexpr int TC = Stage32<Q>::TC;
        int ncnt[NT];  // entries in this warp's list of each slot (warp-uniform)
#pragma unroll
        for (int s = 0; s < NT; ++s) ncnt[s] = 0;
        // evaluate the listed near pairs of slot s (lane i takes entry i), sum over the
        // warp in butterfly order, lane 0 adds the batch to R.N
        auto flush = [&](int s) {
            double d[4] = {0.0, 0.0, 0.0, 0.0};
            if (lane < ncnt[s]) near_pair(s, R.near[warp][s][lane], d);
#pragma unroll
            for (int c = 0; c < 4; ++c) d[c] = wsum(d[c]);
            if (lane == 0)
#pragma unroll
                for (int c = 0; c < 4; ++c) R.N[tk[s]][warp][c] += d[c];
            __syncwarp();
            ncnt[s] = 0;
        };
        constexpr int NS = Stage32<Q>::NS;
        constexpr int GW = TC / 32;
        const RankGroups RG(A.np, rank, ncl);
        const int64_t nch = (RG.ngroups + GW - 1) / GW;
        const int t = threadIdx.x;
        // prologue: chunks 0 .. NS-2 in flight (one commit group per chunk, empty past the end);
        // the previous round's reads of the ring ended before the round's entry barrier
#pragma unroll
        for (int p = 0; p < NS - 1; ++p) {
            if (p < nch) stage_chunk<Q>(A, S, p, RG, p);
            cp_async_commit();
        }
        for (int64_t c = 0; c < nch; ++c) {
            const int b = (int)(c % NS);
            cp_async_wait<NS - 2>();  // this lane's copies of chunks 0..c have landed (NS-2 newer groups may be in flight)
            __syncwarp();             // ... for every lane of the warp; and every lane is done with chunk c-1
            const int64_t cn = c + NS - 1;  // its buffer, (c-1) % NS, takes chunk c+NS-1 now
            if (cn < nch) stage_chunk<Q>(A, S, (int)(cn % NS), RG, cn);
            cp_async_commit();
            const int64_t g0 = warp < GW ? RG.first(c * GW + warp) : -1;
            const int64_t j = g0 + lane;
            const bool valid = t < TC && g0 >= 0 && j < A.np;
            bool nearf[NT];
            if (valid) {
                const float4 nv = S.nrm[b][t];
                const float4 h = S.hdr[b][t];
                const int rj = __float_as_int(nv.w);
                const bool elec = A.electrode[rj] != 0;
                const float uf = S.u[b][t];
                float gx[NT], gy[NT], gz[NT];
                if constexpr (NT >= 2) {
                    // two points per paired FP32 instruction (the same operations per lane,
                    // so the sums are those of the scalar loop below, bit for bit)
                    float2 ax[NT / 2], ay[NT / 2], az[NT / 2];
#pragma unroll
                    for (int s = 0; s < NT / 2; ++s) ax[s] = ay[s] = az[s] = make_float2(0.f, 0.f);
                    const float2 eps2 = make_float2(1e-20f, 1e-20f);
#pragma unroll
                    for (int q = 0; q < Q; ++q) {
                        const float4 nd = S.node[b][t * Q + q];
                        const float2 mx = make_float2(-nd.x, -nd.x), my = make_float2(-nd.y, -nd.y),
                                     mz = make_float2(-nd.z, -nd.z), w2 = make_float2(nd.w, nd.w);
#pragma unroll
                        for (int s = 0; s < NT / 2; ++s) {
                            const float2 dx = __fadd2_rn(x2[s], mx), dy = __fadd2_rn(y2[s], my),
                                         dz = __fadd2_rn(z2[s], mz);
                            const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, eps2)));
                            const float2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
                            const float2 t3 = __fmul2_rn(__fmul2_rn(__fmul2_rn(w2, ri), ri), ri);
                            ax[s] = __ffma2_rn(t3, dx, ax[s]);
                            ay[s] = __ffma2_rn(t3, dy, ay[s]);
                            az[s] = __ffma2_rn(t3, dz, az[s]);
                        }
                    }
#pragma unroll
                    for (int s = 0; s < NT / 2; ++s) {
                        gx[2 * s] = ax[s].x; gx[2 * s + 1] = ax[s].y;
                        gy[2 * s] = ay[s].x; gy[2 * s + 1] = ay[s].y;
                        gz[2 * s] = az[s].x; gz[2 * s + 1] = az[s].y;
                    }
                } else {
#pragma unroll
                    for (int s = 0; s < NT; ++s) gx[s] = gy[s] = gz[s] = 0.f;
#pragma unroll
                    for (int q = 0; q < Q; ++q) {
                        const float4 nd = S.node[b][t * Q + q];
#pragma unroll
                        for (int s = 0; s < NT; ++s) {
                            const float dx = xf[s] - nd.x, dy = yf[s] - nd.y, dz = zf[s] - nd.z;
                            const float ri = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, 1e-20f))));
                            const float t3 = nd.w * ri * ri * ri;
                            gx[s] = fmaf(t3, dx, gx[s]); gy[s] = fmaf(t3, dy, gy[s]); gz[s] = fmaf(t3, dz, gz[s]);
                        }
                    }
                }
#pragma unroll
                for (int s = 0; s < NT; ++s) {
                    const bool far = is_far32(xf[s], yf[s], zf[s], h);
                    nearf[s] = !far && s < nt;
                    const float m = far ? uf : 0.f;
                    fx[s] = fmaf(m, gx[s], fx[s]); fy[s] = fmaf(m, gy[s], fy[s]); fz[s] = fmaf(m, gz[s], fz[s]);
                    if (far && elec && rj != sr[s])
                        fi[s] = fmaf(gz[s], nv.z, fmaf(gy[s], nv.y, fmaf(gx[s], nv.x, fi[s])));
                }
            } else {
#pragma unroll
                for (int s = 0; s < NT; ++s) nearf[s] = false;
            }
            // list the near pairs (the warp is converged here)
#pragma unroll
            for (int s = 0; s < NT; ++s) {
                const unsigned bal = __ballot_sync(0xffffffffu, nearf[s]);
                if (bal == 0u) continue;
                const int cnt = __popc(bal);
                if (ncnt[s] + cnt > kNearCap) flush(s);
                if (nearf[s]) R.near[warp][s][ncnt[s] + __popc(bal & ((1u << lane) - 1u))] = (int32_t)j;
                __syncwarp();
                ncnt[s] += cnt;
            }
        }
        cp_async_wait<0>();  // no copies left in flight (the trailing groups are empty)
#pragma unroll
        for (int s = 0; s < NT; ++s)
            if (ncnt[s] > 0) flush(s);
        // per-slot warp sums of the regular pairs (fixed butterfly order)
#pragma unroll
        for (int s = 0; s < NT; ++s) {
            if (s >= nt) continue;
            const float a = wsumf(fx[s]), bb = wsumf(fy[s]), cc = wsumf(fz[s]), dd = wsumf(fi[s]);
            if (lane == 0) {
                const int k = tk[s];
                R.F[k][warp][0] = a; R.F[k][warp][1] = bb; R.F[k][warp][2] = cc; R.F[k][warp][3] = dd;
                R.G[k][warp][0] = R.G[k][warp][1] = R.G[k][warp][2] = R.G[k][warp][3] = 0.0;
            }
        }
    } else {
        int64_t j0, j1;
        rank_range(A.np, rank, ncl, j0, j1);
        for (int s = 0; s < nt; ++s) {
            const int k = (int)__fns(amask, 0, s + 1);
            const double* xs = R.x[k];
            const int srk = R.sr[k];
            double q[4] = {0.0, 0.0, 0.0, 0.0}, d[4] = {0.0, 0.0, 0.0, 0.0};
            for (int64_t j = j0 + threadIdx.x; j < j1; j += kLT) {
                if (is_far64(xs[0], xs[1], xs[2], A.hdr64[j])) {
                    const int rj = A.region[j];
                    const double* gp = A.geo + GEO_STRIDE * j;
                    const double uj = A.u[j];
                    double gx = 0.0, gy = 0.0, gz = 0.0;
#pragma unroll
                    for (int qq = 0; qq < Q; ++qq) {
                        const double4 nd = A.node64[j * Q + qq];
                        const double dx = xs[0] - nd.x, dy = xs[1] - nd.y, dz = xs[2] - nd.z;
                        const double ri = rsqrt(fma(dx, dx, fma(dy, dy, fma(dz, dz, 1e-200))));
                        const double t3 = nd.w * ri * ri * ri;
                        gx = fma(t3, dx, gx); gy = fma(t3, dy, gy); gz = fma(t3, dz, gz);
                    }
                    q[0] = fma(uj, gx, q[0]); q[1] = fma(uj, gy, q[1]); q[2] = fma(uj, gz, q[2]);
                    if (A.electrode[rj] != 0 && rj != srk) q[3] += gx * gp[GEO_N] + gy * gp[GEO_N + 1] + gz * gp[GEO_N + 2];
                } else {
                    // near pair in place (slot index of k is s)
                    const double* gp = A.geo + GEO_STRIDE * j;
                    const int rj = A.region[j];
                    const double uj = A.u[j];
                    double S, Gx, Gy, Gz;
                    tri_closed_form(gp, xs[0], xs[1], xs[2], false, S, Gx, Gy, Gz);
                    d[0] = fma(uj, Gx, d[0]); d[1] = fma(uj, Gy, d[1]); d[2] = fma(uj, Gz, d[2]);
                    if (A.electrode[rj] != 0 && rj != srk) d[3] += Gx * gp[GEO_N] + Gy * gp[GEO_N + 1] + Gz * gp[GEO_N + 2];
                }
            }
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                q[c] = wsum(q[c]);
                d[c] = wsum(d[c]);
            }
            if (lane == 0)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    R.F[k][warp][c] = 0.f;
                    R.G[k][warp][c] = q[c];
                    R.N[k][warp][c] = d[c];
                }
        }
    }
}

// This CTA's part of the field at every posted point: the triangles of cluster rank
// `rank` of ncl (RankGroups in the FP32 form, rank_range in the FP64 form), the
// variant for the number of posting warps, rounded up to 1, 2, 4 or 8.
template <bool F32, int Q>
__device__ __noinline__ void sweep(const TArgs& A, Round& R, int rank, int ncl)
{
    unsigned amask = 0u;
#pragma unroll
    for (int k = 0; k < kLW; ++k)
        if (R.act[k]) amask |= 1u << k;
    const int nt = __popc(amask);
    if (nt == 0) return;
    if constexpr (!F32) {
        eval_targets<F32, Q, 1>(A, R, amask, nt, rank, ncl);  // the FP64 form loops over the slots
    } else if (nt == 1) {
        eval_targets<F32, Q, 1>(A, R, amask, nt, rank, ncl);
    } else if (nt == 2) {
        eval_targets<F32, Q, 2>(A, R, amask, nt, rank, ncl);
    } else if (nt <= 4) {
        eval_targets<F32, Q, 4>(A, R, amask, nt, rank, ncl);
    } else {
        eval_targets<F32, Q, 8>(A, R, amask, nt, rank, ncl);
    }
}

// A round of the cluster, on the leader (all its threads call this after the round's
// entry barrier, with at least one point posted): push the posted points and the
// arguments into every helper's round, meet the helpers at the cluster barrier,
// sweep the leader's part of the triangles, and meet them again -- by then every
// helper has left its part in its own R.P.
template <bool F32, int Q>
__device__ void eval_round(const TArgs& A, Round& R)
{
    cg::cluster_group cl = cg::this_cluster();
    const int ncl = (int)cl.num_blocks();
    for (int h = 1; h < ncl; ++h) {
        Round* Rh = cl.map_shared_rank(&R, h);
        for (int i = threadIdx.x; i < kLW * 3; i += kLT) Rh->x[i / 3][i % 3] = R.x[i / 3][i % 3];
        if (threadIdx.x < kLW) {
            Rh->sr[threadIdx.x] = R.sr[threadIdx.x];
            Rh->act[threadIdx.x] = R.act[threadIdx.x];
        }
        if (threadIdx.x == 0) {
            Rh->args = A;
            Rh->exit = 0;
        }
    }
    cl.sync();
    sweep<F32, Q>(A, R, 0, ncl);
    cl.sync();
}

// The leader's last act: the helpers leave their loop.
__device__ __forceinline__ void release_helpers(Round& R)
{
    cg::cluster_group cl = cg::this_cluster();
    if (threadIdx.x == 0)
        for (int h = 1; h < (int)cl.num_blocks(); ++h) cl.map_shared_rank(&R, h)->exit = 1;
    cl.sync();
}

// A helper CTA (cluster rank >= 1): one iteration per round of its leader -- wait for
// the pushed round, sweep this rank's part of the triangles for the posted points,
// sum the warps' partial sums into R.P, meet the leader again.  Its barriers pair one
// to one with the leader's (two per round, one at the release), so every CTA of the
// cluster goes through the same sequence of cluster barriers.  The leader writes a
// helper's x, sr, act, args and exit only between the helper's second barrier of a
// round and its first of the next (the helper reads them after that one), and reads
// a helper's P only between those two barriers too (the helper writes it before the
// second), so no access races.
template <bool F32, int Q>
__device__ void helper_rounds(Round& R, int rank)
{
    cg::cluster_group cl = cg::this_cluster();
    for (;;) {
        cl.sync();                    // the leader has pushed a round, or the release
        if (R.exit) break;
        sweep<F32, Q>(R.args, R, rank, (int)cl.num_blocks());
        cta_bar();                    // every warp's partial sums are in R
        for (int i = threadIdx.x; i < kLW * 12; i += kLT) {
            const int k = i / 12, a = (i % 12) / 4, c = i % 4;
            if (!R.act[k]) continue;
            double v = 0.0;
#pragma unroll
            for (int u = 0; u < kLW; ++u) v += a == 0 ? (double)R.F[k][u][c] : (a == 1 ? R.N[k][u][c] : R.G[k][u][c]);
            R.P[k][i % 12] = v;
        }
        cl.sync();                    // the leader may read R.P
    }
}

// the field at warp w's point from the round's partial sums: lane 4a+c (a = 0 FP32
// regular pairs, 1 closed-form pairs, 2 FP64 regular pairs; c = component) adds its
// sum over the warps in order, and the twelve sums reach every lane by shuffles
// (one FP64 add per warp and lane instead of twelve)
__device__ __forceinline__ V4 round_result(const Round& R, int w)
{
    const int lane = threadIdx.x & 31;
    const int a = min(lane >> 2, 2), c = lane & 3;
    double v = 0.0;
#pragma unroll
    for (int u = 0; u < kLW; ++u)
        v += a == 0 ? (double)R.F[w][u][c] : (a == 1 ? R.N[w][u][c] : R.G[w][u][c]);
    // the helpers' parts, in rank order
    cg::cluster_group cl = cg::this_cluster();
    const int ncl = (int)cl.num_blocks();
    for (int h = 1; h < ncl; ++h) v += cl.map_shared_rank(&R, h)->P[w][4 * a + c];
    double f[4], n[4], g[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        f[k] = __shfl_sync(0xffffffffu, v, k);
        n[k] = __shfl_sync(0xffffffffu, v, 4 + k);
        g[k] = __shfl_sync(0xffffffffu, v, 8 + k);
    }
    return V4{n[0] + kInv4Pi * (g[0] + f[0]), n[1] + kInv4Pi * (g[1] + f[1]),
              n[2] + kInv4Pi * (g[2] + f[2]), n[3] + kInv4Pi * (g[3] + f[3])};
}

// The calling warp's field at x (all 32 lanes call this with the same x): one round.
template <bool F32, int Q>
__device__ V4 field(const TArgs& A, Round& R, const double* x, int seed_region)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        R.x[w][0] = x[0]; R.x[w][1] = x[1]; R.x[w][2] = x[2];
        R.sr[w] = seed_region;
        R.act[w] = 1;
    }
    cta_bar();
    eval_round<F32, Q>(A, R);
    cta_bar();
    return round_result(R, w);
}

// A round in which the calling warp posts nothing; false if no warp posted a point
// (then every warp of the CTA is in this round and returns false from it).  *exh
// receives the CTA's "no lines left" flag as it stands during the round: warps
// change that flag only outside rounds, so in a round without posted points every
// warp reads the same value.
template <bool F32, int Q>
__device__ bool idle_round(const TArgs& A, Round& R, const int* flag, int& exh)
{
    if ((threadIdx.x & 31) == 0) R.act[threadIdx.x >> 5] = 0;
    cta_bar();
    bool any = false;
#pragma unroll
    for (int k = 0; k < kLW; ++k) any = any || R.act[k] != 0;
    exh = *(const volatile int*)flag;
    if (any) eval_round<F32, Q>(A, R);
    cta_bar();
    return any;
}

__device__ __forceinline__ double norm3(double a, double b, double c) { return sqrt(a * a + b * b + c * c); }

__device__ __forceinline__ double alpha_eff(const TArgs& A, double Em, int side)
{
    return side > 0 ? A.c * (Em - A.E0) * (Em - A.E0) : -A.d;
}

// one RK4 step of length s from (x, K); E0c: field at x if known
template <bool F32, int Q>
__device__ void rk4(const TArgs& A, Round& R, int seed_region, double s0, int side, const double* x,
                    double K, double s, const V4* E0c, double* x1, double& K1)
{
    double k[4][3], a[4], y[3] = {x[0], x[1], x[2]};
    for (int st = 0; st < 4; ++st) {
        const V4 E = (st == 0 && E0c) ? *E0c : field<F32, Q>(A, R, y, seed_region);
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
__device__ double event_g(const TArgs& A, Round& R, int seed_region, double s0, int side, const double* x,
                          double K, const V4* E0c, double sig, int ev)
{
    double x1[3], K1;
    rk4<F32, Q>(A, R, seed_region, s0, side, x, K, sig, E0c, x1, K1);
    if (ev == EV_RMAX) return norm3(x1[0], x1[1], x1[2]) - A.r_max;
    const V4 E = field<F32, Q>(A, R, x1, seed_region);
    if (ev == EV_ALPHA) return norm3(E.x, E.y, E.z) - A.E0;
    return E.w + 0.5;
}

// Illinois regula falsi for the root of an event function g on [0, b], g(0) = ga,
// g(b) = gb.  The event is detected at the end of the step (gb on the far side, or
// zero: a root at b); if ga is already on that side (or zero) the condition held
// where the sub-step starts and there is no crossing inside: the event is at 0.
template <bool F32, int Q>
__device__ double illinois(const TArgs& A, Round& R, int seed_region, double s0, int side, const double* x,
                           double K, const V4* E0c, double b, double ga, double gb, int ev)
{
    if (gb == 0.0) return b;
    if (ga == 0.0 || (ga > 0.0) == (gb > 0.0)) return 0.0;
    double a = 0.0, c = b;
    int last = 0;
    for (int it = 0; it < 100; ++it) {
        c = (ga * b - gb * a) / (ga - gb);
        const double gc = event_g<F32, Q>(A, R, seed_region, s0, side, x, K, E0c, c, ev);
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

// The steps [step0, step_end) of a line (capped at max_steps) from the state at the
// start of step0: point x, integral K, branch side, direction s0 and seed region.
// The field at x is evaluated afresh, as at every step start after an event, so a
// line resumed from a state recorded at a step start continues bit for bit as the
// uninterrupted line (a line's arithmetic does not depend on the lines sharing its
// rounds).  Status 3 (step limit) is returned when step_end is reached; the caller
// that resumes knows whether that was a segment's end or the line's.
template <bool F32, int Q, class Rec>
__device__ void trace_steps(const TArgs& A, Round& R, double* x, double& K, int side, double s0,
                            int seed_region, int64_t step0, int64_t step_end, Rec& rec, int& st_out,
                            int64_t& ns_out)
{
    V4 E;
    int st = 3;
    int64_t step = step0;
    bool have = false;  // E holds the field at x (with the seed's indicator)
    const int64_t last = min(step_end, A.max_steps);
    for (; step < last; ++step) {
        if (!have) E = field<F32, Q>(A, R, x, seed_region);
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
            rk4<F32, Q>(A, R, seed_region, s0, side, x, K, rem, Ec, x1, K1);
            const V4 E1 = field<F32, Q>(A, R, x1, seed_region);
            const double E1m = norm3(E1.x, E1.y, E1.z);
            double best = 2.0 * rem;
            int which = -1;
            if ((E1m > A.E0) != (side > 0)) {
                const double ga = event_g<F32, Q>(A, R, seed_region, s0, side, x, K, Ec, 0.0, EV_ALPHA);
                const double sg = illinois<F32, Q>(A, R, seed_region, s0, side, x, K, Ec, rem, ga, E1m - A.E0, EV_ALPHA);
                if (sg < best) { best = sg; which = EV_ALPHA; }
            }
            const double r1 = norm3(x1[0], x1[1], x1[2]);
            if (r1 >= A.r_max) {
                const double sg = illinois<F32, Q>(A, R, seed_region, s0, side, x, K, Ec, rem,
                                                   norm3(x[0], x[1], x[2]) - A.r_max, r1 - A.r_max, EV_RMAX);
                if (sg < best) { best = sg; which = EV_RMAX; }
            }
            if (E1.w < -0.5) {
                const double ga = event_g<F32, Q>(A, R, seed_region, s0, side, x, K, Ec, 0.0, EV_ELECTRODE);
                const double sg = illinois<F32, Q>(A, R, seed_region, s0, side, x, K, Ec, rem, ga, E1.w + 0.5, EV_ELECTRODE);
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
            rk4<F32, Q>(A, R, seed_region, s0, side, x, K, best, Ec, xn, Kn);
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
    st_out = st;
    ns_out = step;
}

// Trace one line from seed xs; the 32 lanes of one warp call this with the same
// arguments while the other warps of the CTA trace their own lines or idle.  The
// outputs (K, status, steps, end point) are returned to every lane.
template <bool F32, int Q, class Rec>
__device__ void trace_line(const TArgs& A, Round& R, const double* xs, Rec& rec, double& K_out,
                           int& st_out, int64_t& ns_out, double* xe_out)
{
    double x[3] = {xs[0], xs[1], xs[2]};
    double K = 0.0;
    // electrode of the seed: the triangle with the nearest centroid (first on ties)
    double bd = 1e300;
    long long bj = 0;
    for (int64_t j = threadIdx.x & 31; j < A.np; j += 32) {
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
    const int seed_region = A.region[bj];
    const double* nb = A.geo + GEO_STRIDE * bj + GEO_N;
    V4 E = field<F32, Q>(A, R, x, -2);
    const double s0 = (E.x * nb[0] + E.y * nb[1] + E.z * nb[2]) >= 0.0 ? 1.0 : -1.0;
    int side = norm3(E.x, E.y, E.z) > A.E0 ? 1 : -1;
    rec.begin(s0, seed_region);
    int st;
    int64_t step;
    trace_steps<F32, Q>(A, R, x, K, side, s0, seed_region, 0, A.max_steps, rec, st, step);
    K_out = K;
    st_out = st;
    ns_out = step;
    xe_out[0] = x[0]; xe_out[1] = x[1]; xe_out[2] = x[2];
}

// Persistent driver: the warps of a tracer CTA take lines of the CTA's current mesh
// from that mesh's counter (next[i], lines 0..L(i)-1) and trace them with
// line_fn(A, R, mesh, line).  A CTA holds at most ceil(total / CTAs) lines at a
// time (1..kLW), so the lines spread over all SMs instead of piling onto the CTAs
// that start first; a warp without a line joins the rounds of the others and tries
// again after each round.  When the mesh's counter has passed L the CTA leaves it
// in the first round in which no warp posts a point (all warps together), and moves
// to another mesh with lines left.  The counters only grow, so the loops end.
// s_int: three shared ints (current mesh, lines held, no-lines-left flag).
// The CTAs of a launch form clusters of 1 or kCl: the leader (rank 0) runs this loop, and
// every round it evaluates is shared with the helpers (eval_round); a helper runs
// helper_rounds until the leader releases it.
template <bool F32, int Q, class ArgsFn, class CountFn, class LineFn>
__device__ void run_lines(ArgsFn args, CountFn L, int ninst, int64_t total, unsigned long long* next,
                          TArgs& sA, Round& R, int* s_int, LineFn line_fn)
{
    const int rank = (int)cg::this_cluster().block_rank();
    if (rank != 0) {
        helper_rounds<F32, Q>(R, rank);
        return;
    }
    const int lane = threadIdx.x & 31;
    const int ncl = (int)cg::this_cluster().num_blocks();
    const int64_t nlead = gridDim.x / ncl;  // clusters of the launch
    const int cap = (int)min((int64_t)kLW, max((int64_t)1, (total + nlead - 1) / nlead));
    int start = (int)((blockIdx.x / ncl) % (unsigned)ninst);
    for (;;) {
        if (threadIdx.x == 0) {
            int pick = -1;
            for (int k = 0; k < ninst; ++k) {
                const int i = (start + k) % ninst;
                if (*(volatile unsigned long long*)&next[i] < (unsigned long long)L(i)) {
                    pick = i;
                    break;
                }
            }
            s_int[0] = pick;
            s_int[1] = 0;
            s_int[2] = 0;
            if (pick >= 0) sA = args(pick);
        }
        cta_bar();
        const int ci = s_int[0];
        if (ci < 0) break;
        const unsigned long long Lc = (unsigned long long)L(ci);
        for (;;) {
            int got = 0;
            unsigned long long l = 0;
            if (lane == 0 && *(volatile int*)&s_int[2] == 0) {
                if (atomicAdd(&s_int[1], 1) < cap) {
                    l = atomicAdd(&next[ci], 1ull);
                    if (l < Lc) {
                        got = 1;
                    } else {
                        atomicExch(&s_int[2], 1);
                        atomicSub(&s_int[1], 1);
                    }
                } else {
                    atomicSub(&s_int[1], 1);
                }
            }
            got = __shfl_sync(0xffffffffu, got, 0);
            l = __shfl_sync(0xffffffffu, l, 0);
            if (got) {
                line_fn(sA, R, ci, (int64_t)l);
                if (lane == 0) atomicSub(&s_int[1], 1);
                continue;
            }
            int exh = 0;
            if (!idle_round<F32, Q>(sA, R, &s_int[2], exh) && exh) break;
        }
        start = ci;
        cta_bar();  // sA and s_int are rewritten next
    }
    release_helpers(R);
}

// persistent grid of a tracer kernel, in whole clusters: as many clusters as the GPU
// holds at once (a cluster must fit in one GPC, so wide clusters may leave SMs
// over), but never more clusters than lines (with the per-cluster cap of run_lines,
// few lines spread one per cluster, many lines fill every warp)
template <class... KArgs>
inline unsigned lines_grid(void (*k)(KArgs...), size_t smem, int num_sms, int64_t lines, int ncl)
{
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kLT, smem) != cudaSuccess) {
        cudaGetLastError();
        per_sm = 1;
    }
    int64_t clusters = (int64_t)num_sms * std::max(per_sm, 1) / ncl;
    if (ncl > 1) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(ncl * clusters));
        cfg.blockDim = dim3(kLT);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = ncl;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, k, &cfg) == cudaSuccess && nc > 0)
            clusters = std::min<int64_t>(clusters, nc);
        else
            cudaGetLastError();
    }
    return (unsigned)(ncl * std::max<int64_t>(1, std::min(clusters, lines)));
}

// launch a tracer kernel as clusters of ncl CTAs (1: plain CTAs)
template <class... KArgs, class... Args>
inline cudaError_t launch_lines(void (*kernel)(KArgs...), unsigned grid, size_t smem, cudaStream_t s, int ncl,
                                Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kLT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = ncl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace tcore

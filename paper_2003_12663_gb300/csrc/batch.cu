// batch.cu -- many meshes of uneven size, up to four right-hand sides each, solved and
// traced together (the operators of Secs. 3-5, scheduled for a family of devices).
//
// * Regular pairs: ONE persistent launch serves every instance.  Its CTAs take work
//   items (instance, tile of 256 targets, slice of triangles) from an atomic counter
//   until the list is exhausted, so meshes of 2k and 30k triangles share the GPU
//   without a launch per mesh.  All instances use the same slice length, so items
//   cost about the same.  An item folds all right-hand sides of its instance into
//   one pass over the quadrature nodes: the node sums of a pair do not depend on the
//   density, only the final multiply does.  The arithmetic per pair is that of the
//   single-mesh FP32 kernel: FP32 node sums, the FP32 classification, per-chunk
//   partials added with Kahan compensation, one FP64 partial per slice.
// * The systems (instance, right-hand side) run restarted GMRES with right Jacobi
//   scaling in lock step.  Hessenberg columns, Givens rotations, residual estimates
//   and the "still iterating" flags live on the device, so one Arnoldi iteration of
//   all systems (scaling, the batched product, two rounds of classical Gram-Schmidt,
//   normalisation, rotation, stop test) is a fixed kernel sequence.  A whole restart
//   cycle, m such iterations, is captured once as a CUDA graph and replayed, its
//   kernels reading the iteration index and the flags from device memory; once no
//   system iterates, the remaining iterations of the cycle do no work.  After each
//   replay the host reads one int (the number of systems still iterating).
// * Iterative refinement as in bem_solve: the correction equations are solved with
//   the FP32 products above, the residual b - A u with each instance's FP64-accurate
//   operator (double-FP32 regular pairs by default).
// * bem_batch_trace: one persistent launch traces the lines of all instances (a CTA
//   takes one line at a time from an atomic counter) with the integrator of
//   bem_trace_lines, so each line's result equals that call's bit for bit.
// No CTA waits for another: the work counters are plain atomicAdd.
#include <algorithm>
#include <cmath>
#include <vector>

#include "trace_core.cuh"

int trace_args(bem_ctx* c, const bem_trace_params* tp, const double* u, tcore::TArgs* out);

namespace {

constexpr int kBT = 128;   // threads per CTA of the batched regular-pair kernel
constexpr int kBTR = 2;    // targets per thread
constexpr int kBPC = 32;   // triangles per shared-memory staging chunk
constexpr int kTile = kBT * kBTR;

struct Inst {  // one mesh, device view
    int64_t np, n, splits, slice;
    const float4* tgt32;
    const float4* hdr32;
    const float4* node32;
    const double* geo;
    const int64_t* near_ptr;
    const int32_t* near_col;
    const double4* near_val;
    const uint8_t* near_flag;
    const int32_t* kind;
    const int32_t* aux;
    const double* ra;
    const double* rb;
    const double* rw;
    const double* rs;
    const double* jinv;
    const int32_t* frows;
    const int32_t* foff;
    int32_t nfloat, pad;
    double* part;  // [nr][splits][np][4] FP64 partial sums of the regular pairs
    double* z;     // [nr][n] the vectors the product multiplies
};

// the vectors of a system; each lives in an instance block [nr][n] at offset rhs * n
enum { V_W = 0, V_Z, V_D, V_R, V_RI, V_B, V_X, V_Y, V_NEUT, NVEC };

struct Sys {
    int32_t inst, rhs;
    int64_t n, np;
    double* vec[NVEC];
    double* V;    // [(m+1)][n] Krylov basis
    double* H;    // [m][m+1] Hessenberg matrix, column-major
    double* cs;   // [m]
    double* sn;   // [m]
    double* g;    // [m+1]
    double* y;    // [m]
    double* ht;   // [m+1] Gram-Schmidt coefficients of the current pass
};

struct SysState {
    int32_t jn, iters;  // columns of the current cycle, Arnoldi iterations so far
    double beta2;       // |r|^2 of the cycle's starting residual
    double tol;         // absolute tolerance of the current correction solve
    double res;         // residual estimate |g_{j+1}|
    double sq;          // squared norm scratch
};

// ---------------------------------------------------------------- regular pairs
// The regular pairs of kBTR targets per thread (tx, ty, tz) with triangles [p0, p1) of
// one mesh, for NR densities z[q * zs + j]: FP32 node sums, the FP32 classification,
// per-chunk partials added with Kahan compensation (acc + cmp carries the sum).
template <int Q, int NR>
__device__ __forceinline__ void bfar_range(const float* tx, const float* ty, const float* tz, int64_t p0,
                                           int64_t p1, const float4* __restrict__ hdr,
                                           const float4* __restrict__ node, const double* __restrict__ z,
                                           int64_t zs, float4* s_hdr, float4* s_node, float (*s_u)[kBPC],
                                           float (&acc)[NR][kBTR][4], float (&cmp)[NR][kBTR][4])
{
    const int tid = threadIdx.x;
#pragma unroll
    for (int q = 0; q < NR; ++q)
#pragma unroll
        for (int r = 0; r < kBTR; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[q][r][c] = cmp[q][r][c] = 0.f;
    for (int64_t c0 = p0; c0 < p1; c0 += kBPC) {
        const int npc = (int)min((int64_t)kBPC, p1 - c0);
        __syncthreads();
        for (int k = tid; k < npc; k += kBT) {
            s_hdr[k] = hdr[c0 + k];
#pragma unroll
            for (int q = 0; q < NR; ++q) s_u[q][k] = __double2float_rn(z[q * zs + c0 + k]);
        }
        for (int k = tid; k < npc * Q; k += kBT) s_node[k] = node[c0 * Q + k];
        __syncthreads();
        float cp[NR][kBTR][4];
#pragma unroll
        for (int q = 0; q < NR; ++q)
#pragma unroll
            for (int r = 0; r < kBTR; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) cp[q][r][c] = 0.f;
        for (int p = 0; p < npc; ++p) {
            float ps[kBTR], gx[kBTR], gy[kBTR], gz[kBTR];
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const float4 nd = s_node[p * Q + k];
#pragma unroll
                for (int r = 0; r < kBTR; ++r) {
                    const float dx = tx[r] - nd.x, dy = ty[r] - nd.y, dz = tz[r] - nd.z;
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, 1e-20f)));
                    const float ri = rsqrtf(r2);
                    const float t = nd.w * ri;
                    const float t3 = t * (ri * ri);
                    if (k == 0) {
                        ps[r] = t;
                        gx[r] = t3 * dx; gy[r] = t3 * dy; gz[r] = t3 * dz;
                    } else {
                        ps[r] += t;
                        gx[r] = fmaf(t3, dx, gx[r]);
                        gy[r] = fmaf(t3, dy, gy[r]);
                        gz[r] = fmaf(t3, dz, gz[r]);
                    }
                }
            }
            const float4 h = s_hdr[p];
#pragma unroll
            for (int r = 0; r < kBTR; ++r) {
                const bool far = is_far32(tx[r], ty[r], tz[r], h);
#pragma unroll
                for (int q = 0; q < NR; ++q) {
                    const float m = far ? s_u[q][p] : 0.f;
                    cp[q][r][0] = fmaf(m, ps[r], cp[q][r][0]);
                    cp[q][r][1] = fmaf(m, gx[r], cp[q][r][1]);
                    cp[q][r][2] = fmaf(m, gy[r], cp[q][r][2]);
                    cp[q][r][3] = fmaf(m, gz[r], cp[q][r][3]);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < NR; ++q)
#pragma unroll
            for (int r = 0; r < kBTR; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float y = cp[q][r][c] - cmp[q][r][c];
                    const float t = acc[q][r][c] + y;
                    cmp[q][r][c] = (t - acc[q][r][c]) - y;
                    acc[q][r][c] = t;
                }
    }
}

// Take work items from the queue: thread 0 draws an item and finds its instance by
// binary search in item_off; returns the item (>= total: none left) to every thread.
__device__ __forceinline__ long long draw_item(unsigned long long* queue, const int64_t* item_off, int ninst,
                                               int64_t total, long long* s_item, int* s_inst, int& inst)
{
    if (threadIdx.x == 0) {
        const long long it = (long long)atomicAdd(queue, 1ull);
        int lo = 0;
        if (it < total) {
            int hi = ninst - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (item_off[mid] <= it) lo = mid; else hi = mid - 1;
            }
        }
        *s_item = it;
        *s_inst = lo;
    }
    __syncthreads();
    const long long item = *s_item;
    inst = *s_inst;
    __syncthreads();  // every thread holds the item before thread 0 takes the next
    return item;
}

template <int Q, int NR>
__global__ void __launch_bounds__(kBT)
k_bfar(const Inst* __restrict__ insts, int ninst, const int64_t* __restrict__ item_off,
       int64_t total, unsigned long long* __restrict__ queue, const int* __restrict__ mask,
       unsigned long long* __restrict__ pairs, const int* __restrict__ live)
{
    __shared__ float4 s_hdr[kBPC];
    __shared__ float4 s_node[kBPC * Q];
    __shared__ float s_u[NR][kBPC];
    __shared__ long long s_item;
    __shared__ int s_inst;
    const int tid = threadIdx.x;
    // inside the Arnoldi graph: once no system iterates, the rest of the cycle's
    // iterations return at once (live = the count of iterating systems)
    if (live && *live == 0) return;
    for (;;) {
        int ii;
        const long long item = draw_item(queue, item_off, ninst, total, &s_item, &s_inst, ii);
        if (item >= total) break;
        bool any = false;
#pragma unroll
        for (int q = 0; q < NR; ++q) any = any || mask[ii * NR + q] != 0;
        if (!any) continue;  // no system of this instance needs the product

        const Inst& I = insts[ii];
        const int64_t np = I.np;
        const int64_t local = item - item_off[ii];
        const int64_t tile = local / I.splits, split = local - tile * I.splits;
        const int64_t base = tile * kTile;
        const int64_t p0 = split * I.slice, p1 = min(np, p0 + I.slice);
        float tx[kBTR], ty[kBTR], tz[kBTR];
#pragma unroll
        for (int r = 0; r < kBTR; ++r) {
            const float4 v = I.tgt32[min(base + r * kBT + tid, np - 1)];
            tx[r] = v.x; ty[r] = v.y; tz[r] = v.z;
        }
        float acc[NR][kBTR][4], cmp[NR][kBTR][4];
        bfar_range<Q, NR>(tx, ty, tz, p0, p1, I.hdr32, I.node32, I.z, I.n, s_hdr, s_node, s_u, acc, cmp);
        if (tid == 0)
            atomicAdd(pairs, (unsigned long long)(min((int64_t)kTile, np - base) * (p1 - p0)));
#pragma unroll
        for (int q = 0; q < NR; ++q)
#pragma unroll
            for (int r = 0; r < kBTR; ++r) {
                const int64_t t = base + r * kBT + tid;
                if (t < np) {
                    double* o = I.part + (((int64_t)q * I.splits + split) * np + t) * 4;
#pragma unroll
                    for (int c = 0; c < 4; ++c) o[c] = (double)acc[q][r][c] - (double)cmp[q][r][c];
                }
            }
    }
}

// Field points of one instance for bem_batch_eval_field (device view).
struct PInst {
    const double* pts;   // [M][3]
    const double* u;     // [>= np]
    const float4* hdr32;
    const float4* node32;
    double* part;        // [splits][M][4]: the context's far workspace
    int64_t M, np, splits, slice;
};

// The regular pairs of every instance's field points in one persistent launch:
// work items (instance, tile of kTile points, slice of triangles).
template <int Q>
__global__ void __launch_bounds__(kBT)
k_bfar_pts(const PInst* __restrict__ insts, int ninst, const int64_t* __restrict__ item_off, int64_t total,
           unsigned long long* __restrict__ queue, unsigned long long* __restrict__ pairs)
{
    __shared__ float4 s_hdr[kBPC];
    __shared__ float4 s_node[kBPC * Q];
    __shared__ float s_u[1][kBPC];
    __shared__ long long s_item;
    __shared__ int s_inst;
    const int tid = threadIdx.x;
    for (;;) {
        int ii;
        const long long item = draw_item(queue, item_off, ninst, total, &s_item, &s_inst, ii);
        if (item >= total) break;
        const PInst& I = insts[ii];
        const int64_t local = item - item_off[ii];
        const int64_t tile = local / I.splits, split = local - tile * I.splits;
        const int64_t base = tile * kTile;
        const int64_t p0 = split * I.slice, p1 = min(I.np, p0 + I.slice);
        float tx[kBTR], ty[kBTR], tz[kBTR];
#pragma unroll
        for (int r = 0; r < kBTR; ++r) {
            const int64_t t = min(base + r * kBT + tid, I.M - 1);
            tx[r] = __double2float_rn(I.pts[3 * t]);
            ty[r] = __double2float_rn(I.pts[3 * t + 1]);
            tz[r] = __double2float_rn(I.pts[3 * t + 2]);
        }
        float acc[1][kBTR][4], cmp[1][kBTR][4];
        bfar_range<Q, 1>(tx, ty, tz, p0, p1, I.hdr32, I.node32, I.u, 0, s_hdr, s_node, s_u, acc, cmp);
        if (tid == 0)
            atomicAdd(pairs, (unsigned long long)(min((int64_t)kTile, I.M - base) * (p1 - p0)));
#pragma unroll
        for (int r = 0; r < kBTR; ++r) {
            const int64_t t = base + r * kBT + tid;
            if (t < I.M) {
                double* o = I.part + ((int64_t)split * I.M + t) * 4;
#pragma unroll
                for (int c = 0; c < 4; ++c) o[c] = (double)acc[0][r][c] - (double)cmp[0][r][c];
            }
        }
    }
}

// Row equations (Eqs. Final1-Final3) of every system: one warp per (system, row); the
// FP32 classification's near pairs in FP64 closed form, as in the single-mesh
// product.  Writes W = A Z and the neutrality summands.
__global__ void k_brows(const Inst* __restrict__ insts, const Sys* __restrict__ sys,
                        const int* __restrict__ mask)
{
    const int s = blockIdx.y;
    if (!mask[s]) return;
    const Sys& S = sys[s];
    const Inst& I = insts[S.inst];
    const int lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t np = I.np;
    if (i >= np) return;
    const double* __restrict__ x = S.vec[V_Z];
    const double* __restrict__ part = I.part + (int64_t)S.rhs * I.splits * np * 4;
    double p = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
    for (int64_t q = lane; q < I.splits; q += 32) {
        const double* v = part + (q * np + i) * 4;
        p += v[0]; ex += v[1]; ey += v[2]; ez += v[3];
    }
    p *= kInv4Pi; ex *= kInv4Pi; ey *= kInv4Pi; ez *= kInv4Pi;
    for (int64_t k = I.near_ptr[i] + lane; k < I.near_ptr[i + 1]; k += 32) {
        if (I.near_flag[k] & 1) {
            const double uj = x[I.near_col[k]];
            const double4 v = I.near_val[k];
            p = fma(uj, v.x, p); ex = fma(uj, v.y, ex); ey = fma(uj, v.z, ey); ez = fma(uj, v.w, ez);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        p += __shfl_xor_sync(0xffffffffu, p, o);
        ex += __shfl_xor_sync(0xffffffffu, ex, o);
        ey += __shfl_xor_sync(0xffffffffu, ey, o);
        ez += __shfl_xor_sync(0xffffffffu, ez, o);
    }
    if (lane != 0) return;
    const double* gp = I.geo + GEO_STRIDE * i;
    const double en = ex * gp[GEO_N] + ey * gp[GEO_N + 1] + ez * gp[GEO_N + 2];
    const int kd = I.kind[i];
    double yi;
    if (kd == BEM_CONDUCTOR) yi = p;                           // Eq. Final1
    else if (kd == BEM_FLOATING) yi = p - x[np + I.aux[i]];   // Eq. Final2
    else yi = I.ra[i] * x[i] + I.rb[i] * en;                  // Eq. Final3
    S.vec[V_W][i] = yi;
    // Eq. Final4 summand (Eq. sheets for the rows of a sheet: rs_i != 0)
    S.vec[V_NEUT][i] = kd == BEM_FLOATING ? I.rw[i] * (0.5 * x[i] + en) + I.rs[i] * x[i] : 0.0;
}

// neutrality rows (Eq. Final4), one block per system, fixed summation order
__global__ void k_bneutral(const Inst* __restrict__ insts, const Sys* __restrict__ sys,
                           const int* __restrict__ mask)
{
    __shared__ double sh[256];
    const int s = blockIdx.x;
    if (!mask[s]) return;
    const Sys& S = sys[s];
    const Inst& I = insts[S.inst];
    const double* neut = S.vec[V_NEUT];
    for (int f = 0; f < I.nfloat; ++f) {
        double a = 0.0;
        for (int k = I.foff[f] + threadIdx.x; k < I.foff[f + 1]; k += blockDim.x) a += neut[I.frows[k]];
        sh[threadIdx.x] = a;
        __syncthreads();
        for (int o = blockDim.x / 2; o > 0; o >>= 1) {
            if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) S.vec[V_W][I.np + f] = sh[0];
        __syncthreads();
    }
}

// ---------------------------------------------------------------- vector kernels
// grid (blocks over the longest system, systems); masked-off systems are skipped

// dst = src (src < 0: dst = 0)
__global__ void k_bcopy(const Sys* sys, const int* mask, int dst, int src)
{
    const int s = blockIdx.y;
    if (!mask[s]) return;
    const Sys& S = sys[s];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < S.n) S.vec[dst][i] = src < 0 ? 0.0 : S.vec[src][i];
}

// dst = a - b
__global__ void k_bdiff(const Sys* sys, const int* mask, int dst, int a, int b)
{
    const int s = blockIdx.y;
    if (!mask[s]) return;
    const Sys& S = sys[s];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < S.n) S.vec[dst][i] = S.vec[a][i] - S.vec[b][i];
}

// dst += src
__global__ void k_badd(const Sys* sys, const int* mask, int dst, int src)
{
    const int s = blockIdx.y;
    if (!mask[s]) return;
    const Sys& S = sys[s];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < S.n) S.vec[dst][i] += S.vec[src][i];
}

// |vec|^2 into st.beta2 (to_beta) or st.sq; one block per system, fixed order
__global__ void k_bsq(const Sys* sys, const int* mask, int src, SysState* st, int to_beta)
{
    __shared__ double sh[256];
    const int s = blockIdx.x;
    if (!mask[s]) return;
    const Sys& S = sys[s];
    const double* v = S.vec[src];
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < S.n; i += blockDim.x) a = fma(v[i], v[i], a);
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (to_beta) st[s].beta2 = sh[0];
        else st[s].sq = sh[0];
    }
}

// ---------------------------------------------------------------- batched GMRES
// Start of a restart cycle: beta = |r|, v_0 = r / beta, g = beta e_0.  The system
// iterates in this cycle iff beta > tol and its iteration budget is not spent.
__global__ void k_bstart(const Sys* sys, const int* mask, SysState* st, int* alive, int m, int max_it)
{
    const int s = blockIdx.y;
    if (!mask[s]) return;
    const Sys& S = sys[s];
    const double beta = sqrt(st[s].beta2);
    const bool go = beta > st[s].tol && st[s].iters < max_it;
    if (blockIdx.x == 0) {
        for (int k = threadIdx.x; k <= m; k += blockDim.x) S.g[k] = k == 0 ? beta : 0.0;
        if (threadIdx.x == 0) {
            alive[s] = go ? 1 : 0;
            st[s].jn = 0;
            st[s].res = beta;
        }
    }
    if (!go) return;
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < S.n) S.V[i] = S.vec[V_R][i] / beta;
}

// z = jinv .* v_j
__global__ void k_bjac(const Inst* insts, const Sys* sys, const int* alive, const int* dj)
{
    const int s = blockIdx.y;
    if (!alive[s]) return;
    const Sys& S = sys[s];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= S.n) return;
    S.vec[V_Z][i] = insts[S.inst].jinv[i] * S.V[(int64_t)(*dj) * S.n + i];
}

// ht[k] = <v_k, w> for k <= j: grid (m+1, systems), blocks past j return at once
__global__ void k_bdots(const Sys* sys, const int* alive, const int* dj)
{
    __shared__ double sh[256];
    const int s = blockIdx.y, k = blockIdx.x;
    if (!alive[s] || k > *dj) return;
    const Sys& S = sys[s];
    const double* v = S.V + (int64_t)k * S.n;
    const double* w = S.vec[V_W];
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < S.n; i += blockDim.x) a = fma(v[i], w[i], a);
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) S.ht[k] = sh[0];
}

// w -= sum_k v_k ht[k]; column j of H = ht (first pass) or += ht (second pass)
__global__ void k_bsub(const Sys* sys, const int* alive, const int* dj, int m, int first)
{
    const int s = blockIdx.y;
    if (!alive[s]) return;
    const Sys& S = sys[s];
    const int j = *dj;
    if (blockIdx.x == 0) {
        double* Hj = S.H + (int64_t)j * (m + 1);
        for (int k = threadIdx.x; k <= j; k += blockDim.x) Hj[k] = first ? S.ht[k] : Hj[k] + S.ht[k];
    }
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= S.n) return;
    double a = S.vec[V_W][i];
    for (int k = 0; k <= j; ++k) a = fma(-S.V[(int64_t)k * S.n + i], S.ht[k], a);
    S.vec[V_W][i] = a;
}

// H[j+1][j] = |w|^2 (k_bgivens takes the square root)
__global__ void k_bnorm(const Sys* sys, const int* alive, const int* dj, int m)
{
    __shared__ double sh[256];
    const int s = blockIdx.x;
    if (!alive[s]) return;
    const Sys& S = sys[s];
    const double* w = S.vec[V_W];
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < S.n; i += blockDim.x) a = fma(w[i], w[i], a);
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int j = *dj;
        S.H[(int64_t)j * (m + 1) + j + 1] = sh[0];
    }
}

// v_{j+1} = w / |w|
__global__ void k_bscale(const Sys* sys, const int* alive, const int* dj, int m)
{
    const int s = blockIdx.y;
    if (!alive[s]) return;
    const Sys& S = sys[s];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= S.n) return;
    const int j = *dj;
    const double nr = sqrt(S.H[(int64_t)j * (m + 1) + j + 1]);
    S.V[(int64_t)(j + 1) * S.n + i] = nr > 0.0 ? S.vec[V_W][i] / nr : 0.0;
}

// The last kernel of an Arnoldi iteration (one block): Givens rotations of column j
// for every iterating system, the residual estimate |g_{j+1}| and the stop test; then
// j += 1 and the count of systems still iterating.
__global__ void k_bgivens(const Sys* sys, int* alive, SysState* st, int nsys, int* dj, int m, int max_it,
                          int* count)
{
    __shared__ int s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const int j = *dj;
    for (int s = threadIdx.x; s < nsys; s += blockDim.x) {
        if (!alive[s]) continue;
        if (j >= m) {  // unreachable with the host's replay bound; kept as a guard
            alive[s] = 0;
            continue;
        }
        const Sys& S = sys[s];
        double* Hj = S.H + (int64_t)j * (m + 1);
        Hj[j + 1] = sqrt(fmax(Hj[j + 1], 0.0));
        for (int k = 0; k < j; ++k) {
            const double t = S.cs[k] * Hj[k] + S.sn[k] * Hj[k + 1];
            Hj[k + 1] = -S.sn[k] * Hj[k] + S.cs[k] * Hj[k + 1];
            Hj[k] = t;
        }
        const double den = hypot(Hj[j], Hj[j + 1]);
        S.cs[j] = den > 0.0 ? Hj[j] / den : 1.0;
        S.sn[j] = den > 0.0 ? Hj[j + 1] / den : 0.0;
        Hj[j] = den;
        Hj[j + 1] = 0.0;
        S.g[j + 1] = -S.sn[j] * S.g[j];
        S.g[j] = S.cs[j] * S.g[j];
        const int it = st[s].iters + 1;
        const double res = fabs(S.g[j + 1]);
        st[s].iters = it;
        st[s].jn = j + 1;
        st[s].res = res;
        if (res <= st[s].tol || den == 0.0 || it >= max_it || j + 1 >= m)
            alive[s] = 0;
        else
            atomicAdd(&s_cnt, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        *count = s_cnt;
        *dj = j + 1;
    }
}

// y = H^{-1} g (upper triangular, jn columns), one thread per system
__global__ void k_bsolve(const Sys* sys, const SysState* st, int nsys, int m)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    const Sys& S = sys[s];
    const int nj = st[s].jn;
    for (int k = nj - 1; k >= 0; --k) {
        double t = S.g[k];
        for (int l = k + 1; l < nj; ++l) t -= S.H[(int64_t)l * (m + 1) + k] * S.y[l];
        const double d = S.H[(int64_t)k * (m + 1) + k];
        S.y[k] = d != 0.0 ? t / d : 0.0;
    }
}

// d += jinv .* (V y) for the systems that iterated in this cycle
__global__ void k_bupdate(const Inst* insts, const Sys* sys, const SysState* st)
{
    const int s = blockIdx.y;
    const int nj = st[s].jn;
    if (nj == 0) return;
    const Sys& S = sys[s];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= S.n) return;
    double a = 0.0;
    for (int k = 0; k < nj; ++k) a = fma(S.V[(int64_t)k * S.n + i], S.y[k], a);
    S.vec[V_D][i] = fma(insts[S.inst].jinv[i], a, S.vec[V_D][i]);
}

__global__ void k_bmask_jn(const SysState* st, int nsys, int* mask)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s < nsys) mask[s] = st[s].jn > 0 ? 1 : 0;
}

// ---------------------------------------------------------------- field lines
// the persistent tracer over all meshes: a CTA traces lines of one mesh at a time
// (per-mesh line counters in next[]), then moves to another mesh with lines left
template <bool F32, int Q>
__global__ void __launch_bounds__(tcore::kLT)
k_btrace(const tcore::TArgs* __restrict__ args, const int64_t* __restrict__ loff, int ninst,
         unsigned long long* __restrict__ next, const double* const* __restrict__ seeds,
         double* const* __restrict__ Kout, int32_t* const* __restrict__ stout,
         int32_t* const* __restrict__ nsout)
{
    __shared__ tcore::Round R;
    __shared__ tcore::TArgs sA;
    __shared__ int s_int[3];
    tcore::run_lines<F32, Q>(
        [&](int i) { return args[i]; }, [&](int i) { return loff[i + 1] - loff[i]; }, ninst, loff[ninst], next, sA,
        R, s_int,
        [&](const tcore::TArgs& a, tcore::Round& r, int i, int64_t l) {
            tcore::NoRec rec;
            double K, xe[3];
            int st;
            int64_t ns;
            tcore::trace_line<F32, Q>(a, r, seeds[i] + 3 * l, rec, K, st, ns, xe);
            if ((threadIdx.x & 31) == 0) {
                if (Kout[i]) Kout[i][l] = K;
                if (stout[i]) stout[i][l] = st;
                if (nsout[i]) nsout[i][l] = (int32_t)ns;
            }
        });
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// resident CTAs per SM of the batched regular-pair kernel (its persistent grid)
int far_blocks_per_sm(int g, int nr)
{
    int v = 0;
    cudaError_t e = cudaErrorInvalidValue;
    switch (g * 8 + nr) {
#define OC(G, QQ, NR) \
    case G * 8 + NR: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, k_bfar<QQ, NR>, kBT, 0); break;
        OC(2, 4, 1) OC(2, 4, 2) OC(2, 4, 3) OC(2, 4, 4)
        OC(3, 9, 1) OC(3, 9, 2) OC(3, 9, 3) OC(3, 9, 4)
        OC(4, 16, 1) OC(4, 16, 2) OC(4, 16, 3) OC(4, 16, 4)
#undef OC
        default: break;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        v = 2;
    }
    return std::max(v, 1);
}

}  // namespace

// ---------------------------------------------------------------- the batch object
struct bem_batch {
    cudaStream_t stream = nullptr;  // private, non-blocking (graph capture needs one)
    cudaStream_t caller = nullptr;  // the contexts' stream
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_t0 = nullptr, ev_t1 = nullptr;
    int ninst = 0, nr = 1, nsys = 0, m = 100, g = 3, max_it = 1000, max_refine = 10, rprec = kPrecDF;
    int num_sms = 1, timing = 0, far_per_sm = 2;
    bool any_float = false;
    int64_t maxn = 0, total_items = 0, slice = 2048;
    std::vector<bem_ctx*> ctx;
    std::vector<Inst> h_inst;
    std::vector<Sys> h_sys;
    std::vector<SysState> h_st;
    Inst* d_inst = nullptr;
    Sys* d_sys = nullptr;
    SysState* d_st = nullptr;
    int64_t* d_item_off = nullptr;
    unsigned long long* d_queue = nullptr;  // work counter of the regular-pair items
    unsigned long long* d_lnext = nullptr;  // [n] line counters of the tracer
    unsigned long long* d_pairs = nullptr;
    int* d_j = nullptr;
    int* d_count = nullptr;
    int* h_count = nullptr;                 // pinned
    int* d_alive = nullptr;
    int* d_mask = nullptr;
    int* d_all = nullptr;
    int* d_upd = nullptr;
    tcore::TArgs* d_targs = nullptr;
    int64_t* d_loff = nullptr;
    void** d_tptr = nullptr;                // [4][n]: seeds, K, status, nsteps
    PInst* d_pinst = nullptr;               // [n] field points of bem_batch_eval_field
    int64_t* d_pitem_off = nullptr;         // [n+1]
    unsigned long long* d_epairs = nullptr; // pairs of the batched field-point launches
    std::vector<void*> allocs;
    cudaGraphExec_t graph = nullptr;
    int graph_kernels = 0;
    bem_batch_counters cnt{};
    std::string err;
};

static int berr(bem_batch* b, int code, const char* msg)
{
    b->err = msg ? msg : "";
    return code;
}

#define BB_TRY(b, call)                                                         \
    do {                                                                        \
        const cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) {                                                \
            (b)->err = std::string(#call) + " failed: " + cudaGetErrorString(e_); \
            return BEM_ERR_CUDA;                                                \
        }                                                                       \
    } while (0)
#define BB_LAUNCH(b)                         \
    do {                                     \
        ++(b)->cnt.kernel_launches;          \
        BB_TRY(b, cudaGetLastError());       \
    } while (0)

static void batch_free(bem_batch* b)
{
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (void* p : b->allocs) cudaFree(p);
    if (b->h_count) cudaFreeHost(b->h_count);
    cudaEvent_t evs[] = {b->ev_in, b->ev_out, b->ev_t0, b->ev_t1};
    for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

template <class T>
static bool dalloc(bem_batch* b, T** p, size_t n)
{
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    b->allocs.push_back(q);
    *p = (T*)q;
    return true;
}

extern "C" int bem_batch_create(bem_batch** out, bem_ctx* const* ctxs, int32_t n, int32_t nrhs, int32_t flags)
{
    if (!out) return BEM_ERR_ARG;
    *out = nullptr;
    if (!ctxs || n < 1 || nrhs < 1 || nrhs > kMaxRhs) return BEM_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        const bem_ctx* c = ctxs[i];
        if (!c || c->p1 || c->device != ctxs[0]->device || c->stream != ctxs[0]->stream || c->g != ctxs[0]->g ||
            c->m != ctxs[0]->m || c->g < 2 || c->g > 4)
            return BEM_ERR_ARG;  // one device, one stream, one far_order in 2..4, one restart length
    }
    bem_batch* b = new bem_batch();
    b->ninst = n;
    b->nr = nrhs;
    b->nsys = n * nrhs;
    b->caller = ctxs[0]->stream;
    b->g = ctxs[0]->g;
    b->m = ctxs[0]->m;
    b->max_it = ctxs[0]->prm.max_iters;
    b->max_refine = ctxs[0]->prm.max_refine;
    b->rprec = ctxs[0]->prm.residual == BEM_RESIDUAL_FP64 ? BEM_FP64 : kPrecDF;
    b->num_sms = std::max(ctxs[0]->num_sms, 1);
    b->timing = flags & 1;
    b->far_per_sm = far_blocks_per_sm(b->g, b->nr);
    b->cnt.n_instances = n;
    b->cnt.nrhs = nrhs;
    if (cudaSetDevice(ctxs[0]->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&b->ev_t0) != cudaSuccess || cudaEventCreate(&b->ev_t1) != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        return BEM_ERR_CUDA;
    }
    for (int i = 0; i < n; ++i) b->ctx.push_back(ctxs[i]);
    // slice length: the largest power of two in [128, 2048] that still gives four or
    // more work items per resident CTA over the whole batch
    for (int64_t sl = 2048; sl >= 128; sl /= 2) {
        int64_t items = 0;
        for (int i = 0; i < n; ++i) items += ((ctxs[i]->np + kTile - 1) / kTile) * ((ctxs[i]->np + sl - 1) / sl);
        b->slice = sl;
        if (items >= 4 * (int64_t)b->num_sms * b->far_per_sm) break;
    }
    const int m = b->m, nr = nrhs;
    std::vector<int64_t> item_off(n + 1, 0);
    bool ok = true;
    for (int i = 0; i < n && ok; ++i) {
        bem_ctx* c = ctxs[i];
        Inst I{};
        I.np = c->np;
        I.n = c->nunk;
        I.slice = b->slice;
        I.splits = std::max<int64_t>(1, (c->np + b->slice - 1) / b->slice);
        I.tgt32 = c->tgt32; I.hdr32 = c->hdr32; I.node32 = c->node32; I.geo = c->geo;
        I.near_ptr = c->near_ptr; I.near_col = c->near_col; I.near_val = c->near_val; I.near_flag = c->near_flag;
        I.kind = c->row_kind; I.aux = c->row_aux; I.ra = c->row_a; I.rb = c->row_b; I.rw = c->row_w;
        I.rs = c->row_s;
        I.jinv = c->jinv;
        I.frows = c->float_rows; I.foff = c->float_off; I.nfloat = c->nfloat;
        ok = dalloc(b, &I.part, (size_t)nr * I.splits * I.np * 4);
        double* blocks[NVEC] = {};
        for (int v = 0; v < NVEC && ok; ++v)
            if (v != V_X && v != V_Y) ok = dalloc(b, &blocks[v], (size_t)nr * I.n);
        if (!ok) break;
        I.z = blocks[V_Z];
        item_off[i + 1] = item_off[i] + ((I.np + kTile - 1) / kTile) * I.splits;
        b->h_inst.push_back(I);
        b->maxn = std::max(b->maxn, I.n);
        b->any_float = b->any_float || I.nfloat > 0;
        for (int r = 0; r < nr && ok; ++r) {
            Sys S{};
            S.inst = i;
            S.rhs = r;
            S.n = I.n;
            S.np = I.np;
            for (int v = 0; v < NVEC; ++v) S.vec[v] = blocks[v] ? blocks[v] + (int64_t)r * I.n : nullptr;
            ok = dalloc(b, &S.V, (size_t)(m + 1) * I.n) && dalloc(b, &S.H, (size_t)m * (m + 1)) &&
                 dalloc(b, &S.cs, m) && dalloc(b, &S.sn, m) && dalloc(b, &S.g, m + 1) &&
                 dalloc(b, &S.y, m) && dalloc(b, &S.ht, m + 1);
            b->h_sys.push_back(S);
        }
    }
    b->total_items = item_off[n];
    const int ns = b->nsys;
    ok = ok && dalloc(b, &b->d_inst, n) && dalloc(b, &b->d_sys, ns) && dalloc(b, &b->d_st, ns) &&
         dalloc(b, &b->d_item_off, n + 1) && dalloc(b, &b->d_queue, 1) && dalloc(b, &b->d_lnext, n) && dalloc(b, &b->d_pairs, 1) &&
         dalloc(b, &b->d_j, 1) && dalloc(b, &b->d_count, 1) && dalloc(b, &b->d_alive, ns) &&
         dalloc(b, &b->d_mask, ns) && dalloc(b, &b->d_all, ns) && dalloc(b, &b->d_upd, ns) &&
         dalloc(b, &b->d_targs, n) && dalloc(b, &b->d_loff, n + 1) && dalloc(b, &b->d_tptr, 4 * (size_t)n) &&
         dalloc(b, &b->d_pinst, n) && dalloc(b, &b->d_pitem_off, n + 1) && dalloc(b, &b->d_epairs, 1);
    if (!ok || cudaMallocHost((void**)&b->h_count, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        return BEM_ERR_NOMEM;
    }
    b->h_st.assign(ns, SysState{});
    std::vector<int> ones(ns, 1);
    if (cudaMemcpy(b->d_inst, b->h_inst.data(), n * sizeof(Inst), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_sys, b->h_sys.data(), ns * sizeof(Sys), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_item_off, item_off.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_all, ones.data(), ns * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_st, b->h_st.data(), ns * sizeof(SysState), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(b->d_pairs, 0, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMemset(b->d_epairs, 0, sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        return BEM_ERR_CUDA;
    }
    *out = b;
    return BEM_OK;
}

extern "C" int bem_batch_destroy(bem_batch* b)
{
    if (!b) return BEM_OK;
    cudaStreamSynchronize(b->stream);
    batch_free(b);
    return BEM_OK;
}

extern "C" const char* bem_batch_last_error(const bem_batch* b) { return b ? b->err.c_str() : "null batch"; }

extern "C" int bem_batch_get_counters(bem_batch* b, bem_batch_counters* out)
{
    if (!b || !out) return BEM_ERR_ARG;
    unsigned long long p = 0, ep = 0;
    BB_TRY(b, cudaStreamSynchronize(b->stream));
    BB_TRY(b, cudaMemcpy(&p, b->d_pairs, sizeof(p), cudaMemcpyDeviceToHost));
    BB_TRY(b, cudaMemcpy(&ep, b->d_epairs, sizeof(ep), cudaMemcpyDeviceToHost));
    b->cnt.pairs = (int64_t)p;
    b->cnt.eval_pairs = (int64_t)ep;
    b->cnt.rhs_pairs = (int64_t)p * b->nr;
    *out = b->cnt;
    return BEM_OK;
}

extern "C" int bem_batch_reset_counters(bem_batch* b)
{
    if (!b) return BEM_ERR_ARG;
    BB_TRY(b, cudaStreamSynchronize(b->stream));
    BB_TRY(b, cudaMemset(b->d_pairs, 0, sizeof(unsigned long long)));
    BB_TRY(b, cudaMemset(b->d_epairs, 0, sizeof(unsigned long long)));
    const int64_t ni = b->cnt.n_instances, nr = b->cnt.nrhs;
    b->cnt = bem_batch_counters{};
    b->cnt.n_instances = ni;
    b->cnt.nrhs = nr;
    return BEM_OK;
}

namespace {

// the batch's stream waits for the contexts' stream ...
int enter(bem_batch* b)
{
    BB_TRY(b, cudaEventRecord(b->ev_in, b->caller));
    BB_TRY(b, cudaStreamWaitEvent(b->stream, b->ev_in, 0));
    return BEM_OK;
}

// ... and the other way round
int leave(bem_batch* b)
{
    BB_TRY(b, cudaEventRecord(b->ev_out, b->stream));
    BB_TRY(b, cudaStreamWaitEvent(b->caller, b->ev_out, 0));
    return BEM_OK;
}

// W = A Z for the systems in mask (FP32 regular pairs, FP64 near pairs); live
// (nullable): device count of iterating systems, 0 skips the regular pairs
int apply(bem_batch* b, const int* mask, bool timed, const int* live = nullptr)
{
    cudaStream_t s = b->stream;
    BB_TRY(b, cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned long long), s));
    const unsigned grid = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>(b->total_items, (int64_t)b->num_sms * b->far_per_sm));
    if (timed) BB_TRY(b, cudaEventRecord(b->ev_t0, s));
    switch (b->g * 8 + b->nr) {
#define BF(G, QQ, NR)                                                                          \
    case G * 8 + NR:                                                                           \
        k_bfar<QQ, NR><<<grid, kBT, 0, s>>>(b->d_inst, b->ninst, b->d_item_off, b->total_items, \
                                             b->d_queue, mask, b->d_pairs, live);              \
        break;
        BF(2, 4, 1) BF(2, 4, 2) BF(2, 4, 3) BF(2, 4, 4)
        BF(3, 9, 1) BF(3, 9, 2) BF(3, 9, 3) BF(3, 9, 4)
        BF(4, 16, 1) BF(4, 16, 2) BF(4, 16, 3) BF(4, 16, 4)
#undef BF
        default: return berr(b, BEM_ERR_ARG, "batched product: far_order must be 2..4");
    }
    BB_LAUNCH(b);
    ++b->cnt.far_launches;
    if (timed) {
        BB_TRY(b, cudaEventRecord(b->ev_t1, s));
        BB_TRY(b, cudaEventSynchronize(b->ev_t1));
        float ms = 0.f;
        BB_TRY(b, cudaEventElapsedTime(&ms, b->ev_t0, b->ev_t1));
        b->cnt.far_ms += ms;
        ++b->cnt.far_timed;
    }
    k_brows<<<dim3(nblk(b->maxn * 32, 128), b->nsys), 128, 0, s>>>(b->d_inst, b->d_sys, mask);
    BB_LAUNCH(b);
    if (b->any_float) {
        k_bneutral<<<b->nsys, 256, 0, s>>>(b->d_inst, b->d_sys, mask);
        BB_LAUNCH(b);
    }
    return BEM_OK;
}

// one Arnoldi iteration of every iterating system: the body of the graph
int arnoldi_iteration(bem_batch* b)
{
    cudaStream_t s = b->stream;
    const int m = b->m, ns = b->nsys;
    const dim3 gv(nblk(b->maxn), ns);
    k_bjac<<<gv, 256, 0, s>>>(b->d_inst, b->d_sys, b->d_alive, b->d_j);
    BB_LAUNCH(b);
    if (int rc = apply(b, b->d_alive, false, b->d_count)) return rc;
    for (int pass = 0; pass < 2; ++pass) {  // classical Gram-Schmidt, twice
        k_bdots<<<dim3(m + 1, ns), 256, 0, s>>>(b->d_sys, b->d_alive, b->d_j);
        BB_LAUNCH(b);
        k_bsub<<<gv, 256, 0, s>>>(b->d_sys, b->d_alive, b->d_j, m, pass == 0);
        BB_LAUNCH(b);
    }
    k_bnorm<<<ns, 256, 0, s>>>(b->d_sys, b->d_alive, b->d_j, m);
    BB_LAUNCH(b);
    k_bscale<<<gv, 256, 0, s>>>(b->d_sys, b->d_alive, b->d_j, m);
    BB_LAUNCH(b);
    k_bgivens<<<1, 256, 0, s>>>(b->d_sys, b->d_alive, b->d_st, ns, b->d_j, m, b->max_it, b->d_count);
    BB_LAUNCH(b);
    return BEM_OK;
}

// The graph of one whole restart cycle: m Arnoldi iterations of every system (the
// kernels read the iteration index and the flags from device memory, and once no
// system iterates the rest of the cycle does no work), then the count of systems
// still iterating copied to the host.  One replay and one synchronisation per cycle.
int ensure_graph(bem_batch* b)
{
    if (b->graph) return BEM_OK;
    const int64_t k0 = b->cnt.kernel_launches, f0 = b->cnt.far_launches;
    BB_TRY(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    int rc = BEM_OK;
    for (int j = 0; j < b->m && !rc; ++j) rc = arnoldi_iteration(b);
    if (!rc) {
        const cudaError_t ec = cudaMemcpyAsync(b->h_count, b->d_count, sizeof(int), cudaMemcpyDeviceToHost,
                                               b->stream);
        if (ec != cudaSuccess) rc = berr(b, BEM_ERR_CUDA, "capture of the count copy failed");
    }
    cudaGraph_t gph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->stream, &gph);
    // captured launches do not run now: they are counted per replay instead
    b->graph_kernels = (int)(b->cnt.kernel_launches - k0);
    b->cnt.kernel_launches = k0;
    b->cnt.far_launches = f0;
    if (rc || e != cudaSuccess) {
        cudaGetLastError();
        if (gph) cudaGraphDestroy(gph);
        return rc ? rc : berr(b, BEM_ERR_CUDA, "stream capture of the Arnoldi iteration failed");
    }
    const cudaError_t ei = cudaGraphInstantiate(&b->graph, gph, 0);
    cudaGraphDestroy(gph);
    if (ei != cudaSuccess) {
        cudaGetLastError();
        b->graph = nullptr;
        return berr(b, BEM_ERR_CUDA, "instantiation of the Arnoldi graph failed");
    }
    return BEM_OK;
}

int pull(bem_batch* b)
{
    BB_TRY(b, cudaMemcpyAsync(b->h_st.data(), b->d_st, b->nsys * sizeof(SysState), cudaMemcpyDeviceToHost,
                              b->stream));
    BB_TRY(b, cudaStreamSynchronize(b->stream));
    return BEM_OK;
}

int push(bem_batch* b)
{
    BB_TRY(b, cudaMemcpyAsync(b->d_st, b->h_st.data(), b->nsys * sizeof(SysState), cudaMemcpyHostToDevice,
                              b->stream));
    BB_TRY(b, cudaStreamSynchronize(b->stream));  // h_st may change right after
    return BEM_OK;
}

int set_mask(bem_batch* b, int* d, const std::vector<int>& h)
{
    BB_TRY(b, cudaMemcpyAsync(d, h.data(), h.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
    BB_TRY(b, cudaStreamSynchronize(b->stream));
    return BEM_OK;
}

// Restarted GMRES(m), right Jacobi scaling, on A D_s = RI_s for the systems with
// need[s] (D starts at 0), to |RI_s - A D_s| <= tol[s].  All systems advance
// together; a converged one stops iterating while the others go on.
int gmres(bem_batch* b, std::vector<int> need, const std::vector<double>& tol)
{
    cudaStream_t s = b->stream;
    const int ns = b->nsys, m = b->m;
    const dim3 gv(nblk(b->maxn), ns);
    if (int rc = ensure_graph(b)) return rc;
    if (int rc = set_mask(b, b->d_mask, need)) return rc;
    k_bcopy<<<gv, 256, 0, s>>>(b->d_sys, b->d_mask, V_D, -1);
    BB_LAUNCH(b);
    k_bcopy<<<gv, 256, 0, s>>>(b->d_sys, b->d_mask, V_R, V_RI);
    BB_LAUNCH(b);
    k_bsq<<<ns, 256, 0, s>>>(b->d_sys, b->d_mask, V_R, b->d_st, 1);
    BB_LAUNCH(b);
    for (;;) {  // ends: every cycle spends >= 1 iteration of a bounded budget, or drops the system
        if (int rc = pull(b)) return rc;
        for (int q = 0; q < ns; ++q) {
            b->h_st[q].tol = tol[q];
            b->h_st[q].jn = 0;
        }
        if (int rc = push(b)) return rc;
        BB_TRY(b, cudaMemsetAsync(b->d_alive, 0, ns * sizeof(int), s));
        k_bstart<<<gv, 256, 0, s>>>(b->d_sys, b->d_mask, b->d_st, b->d_alive, m, b->max_it);
        BB_LAUNCH(b);
        BB_TRY(b, cudaMemsetAsync(b->d_j, 0, sizeof(int), s));
        BB_TRY(b, cudaMemsetAsync(b->d_count, 1, sizeof(int), s));  // nonzero: the cycle starts
        // one replay runs the whole cycle; k_bgivens stops every system by j = m
        BB_TRY(b, cudaGraphLaunch(b->graph, s));
        BB_TRY(b, cudaStreamSynchronize(s));
        ++b->cnt.graph_launches;
        b->cnt.kernel_launches += b->graph_kernels;
        b->cnt.far_launches += m;
        k_bsolve<<<nblk(ns, 128), 128, 0, s>>>(b->d_sys, b->d_st, ns, m);
        BB_LAUNCH(b);
        k_bupdate<<<gv, 256, 0, s>>>(b->d_inst, b->d_sys, b->d_st);
        BB_LAUNCH(b);
        k_bmask_jn<<<nblk(ns, 128), 128, 0, s>>>(b->d_st, ns, b->d_upd);
        BB_LAUNCH(b);
        // the true residual of the restart: R = RI - A D
        k_bcopy<<<gv, 256, 0, s>>>(b->d_sys, b->d_upd, V_Z, V_D);
        BB_LAUNCH(b);
        if (int rc = apply(b, b->d_upd, false)) return rc;
        k_bdiff<<<gv, 256, 0, s>>>(b->d_sys, b->d_upd, V_R, V_RI, V_W);
        BB_LAUNCH(b);
        k_bsq<<<ns, 256, 0, s>>>(b->d_sys, b->d_upd, V_R, b->d_st, 1);
        BB_LAUNCH(b);
        if (int rc = pull(b)) return rc;
        bool any = false;
        for (int q = 0; q < ns; ++q) {
            const SysState& t = b->h_st[q];
            need[q] = need[q] && t.jn > 0 && std::sqrt(t.beta2) > tol[q] && t.iters < b->max_it;
            any = any || need[q];
        }
        if (!any) return BEM_OK;
        if (int rc = set_mask(b, b->d_mask, need)) return rc;
    }
}

// point V_X / V_Y of every system at the caller's vectors (instance blocks [nr][n])
int set_user_vectors(bem_batch* b, const double* const* xs, double* const* ys)
{
    for (int q = 0; q < b->nsys; ++q) {
        Sys& S = b->h_sys[q];
        S.vec[V_X] = xs ? const_cast<double*>(xs[S.inst]) + (int64_t)S.rhs * S.n : nullptr;
        S.vec[V_Y] = ys ? ys[S.inst] + (int64_t)S.rhs * S.n : nullptr;
    }
    BB_TRY(b, cudaMemcpyAsync(b->d_sys, b->h_sys.data(), b->nsys * sizeof(Sys), cudaMemcpyHostToDevice, b->stream));
    BB_TRY(b, cudaStreamSynchronize(b->stream));
    return BEM_OK;
}

}  // namespace

extern "C" int bem_batch_matvec(bem_batch* b, const double* const* x, double* const* y)
{
    if (!b) return BEM_ERR_ARG;
    if (!x || !y) return berr(b, BEM_ERR_ARG, "bem_batch_matvec: NULL pointer array");
    for (int i = 0; i < b->ninst; ++i)
        if (!x[i] || !y[i]) return berr(b, BEM_ERR_ARG, "bem_batch_matvec: NULL vector");
    if (int rc = enter(b)) return rc;
    if (int rc = set_user_vectors(b, x, y)) return rc;
    cudaStream_t s = b->stream;
    const dim3 gv(nblk(b->maxn), b->nsys);
    k_bcopy<<<gv, 256, 0, s>>>(b->d_sys, b->d_all, V_Z, V_X);
    BB_LAUNCH(b);
    if (int rc = apply(b, b->d_all, b->timing != 0)) return rc;
    k_bcopy<<<gv, 256, 0, s>>>(b->d_sys, b->d_all, V_Y, V_W);
    BB_LAUNCH(b);
    return leave(b);
}

extern "C" int bem_batch_solve(bem_batch* b, int32_t precision, const double* const* V0, double* const* u,
                               double tol, int32_t* iters, double* relres)
{
    if (!b) return BEM_ERR_ARG;
    if (precision != BEM_MIXED)
        return berr(b, BEM_ERR_ARG, "bem_batch_solve: precision must be BEM_MIXED");
    if (!u || !(tol > 0.0)) return berr(b, BEM_ERR_ARG, "bem_batch_solve: need u != NULL and tol > 0");
    if (!V0 && b->nr != 1) return berr(b, BEM_ERR_ARG, "bem_batch_solve: V0 = NULL needs nrhs = 1");
    for (int i = 0; i < b->ninst; ++i)
        if (!u[i] || (V0 && !V0[i])) return berr(b, BEM_ERR_ARG, "bem_batch_solve: NULL vector");
    const int ns = b->nsys, nr = b->nr;
    cudaStream_t s = b->stream;
    const dim3 gv(nblk(b->maxn), ns);
    // right-hand sides, on the contexts' stream, into the B blocks
    for (int i = 0; i < b->ninst; ++i) {
        bem_ctx* c = b->ctx[i];
        const int rc = bem_rhs(c, nr, V0 ? V0[i] : nullptr, b->h_sys[(size_t)i * nr].vec[V_B]);
        if (rc) return berr(b, rc, bem_last_error(c));
    }
    if (int rc = enter(b)) return rc;
    if (int rc = set_user_vectors(b, u, nullptr)) return rc;
    k_bcopy<<<gv, 256, 0, s>>>(b->d_sys, b->d_all, V_X, -1);
    BB_LAUNCH(b);
    k_bcopy<<<gv, 256, 0, s>>>(b->d_sys, b->d_all, V_RI, V_B);
    BB_LAUNCH(b);
    k_bsq<<<ns, 256, 0, s>>>(b->d_sys, b->d_all, V_B, b->d_st, 0);
    BB_LAUNCH(b);
    if (int rc = pull(b)) return rc;
    std::vector<double> bnorm(ns), rnorm(ns), itol(ns);
    for (int q = 0; q < ns; ++q) {
        bnorm[q] = rnorm[q] = std::sqrt(b->h_st[q].sq);
        b->h_st[q].iters = 0;
    }
    if (int rc = push(b)) return rc;
    std::vector<int> need(ns), inst_need(b->ninst);
    for (int refine = 0; refine < b->max_refine; ++refine) {
        if (int rc = pull(b)) return rc;
        bool any = false;
        std::fill(inst_need.begin(), inst_need.end(), 0);
        for (int q = 0; q < ns; ++q) {
            need[q] = bnorm[q] > 0.0 && rnorm[q] > tol * bnorm[q] && b->h_st[q].iters < b->max_it;
            // correction accuracy: 1e-5 of the current residual (FP32 regular pairs limit it near 1e-7)
            itol[q] = std::max(1e-5 * rnorm[q], 0.5 * tol * bnorm[q]);
            any = any || need[q];
            if (need[q]) inst_need[q / nr] = 1;
        }
        if (!any) break;
        if (int rc = gmres(b, need, itol)) return rc;
        if (int rc = set_mask(b, b->d_mask, need)) return rc;
        k_badd<<<gv, 256, 0, s>>>(b->d_sys, b->d_mask, V_X, V_D);
        BB_LAUNCH(b);
        // residual b - A u with the FP64-accurate operator, per instance on the contexts' stream
        if (int rc = leave(b)) return rc;
        for (int i = 0; i < b->ninst; ++i) {
            if (!inst_need[i]) continue;
            bem_ctx* c = b->ctx[i];
            const int rc = matvec_impl(c, b->rprec, nr, u[i], b->h_sys[(size_t)i * nr].vec[V_W]);
            if (rc) return berr(b, rc, bem_last_error(c));
        }
        if (int rc = enter(b)) return rc;
        k_bdiff<<<gv, 256, 0, s>>>(b->d_sys, b->d_mask, V_RI, V_B, V_W);
        BB_LAUNCH(b);
        k_bsq<<<ns, 256, 0, s>>>(b->d_sys, b->d_mask, V_RI, b->d_st, 0);
        BB_LAUNCH(b);
        if (int rc = pull(b)) return rc;
        for (int q = 0; q < ns; ++q)
            if (need[q]) rnorm[q] = std::sqrt(b->h_st[q].sq);
    }
    bool conv = true;
    for (int q = 0; q < ns; ++q) {
        if (iters) iters[q] = b->h_st[q].iters;
        if (relres) relres[q] = bnorm[q] > 0.0 ? rnorm[q] / bnorm[q] : 0.0;
        b->cnt.arnoldi_steps += b->h_st[q].iters;
        conv = conv && (bnorm[q] == 0.0 || rnorm[q] <= tol * bnorm[q]);
    }
    if (int rc = leave(b)) return rc;
    if (!conv) return berr(b, BEM_ERR_NOT_CONVERGED, "tolerance not reached within the iteration limit");
    return BEM_OK;
}

extern "C" int bem_batch_trace(bem_batch* b, int32_t precision, const double* const* u, const int64_t* L,
                               const double* const* seeds, const bem_trace_params* tp, double* const* K,
                               int32_t* const* status, int32_t* const* nsteps)
{
    if (!b) return BEM_ERR_ARG;
    if (precision != BEM_FP64 && precision != BEM_MIXED)
        return berr(b, BEM_ERR_ARG, "precision must be BEM_FP64 or BEM_MIXED");
    if (!u || !L || !seeds) return berr(b, BEM_ERR_ARG, "bem_batch_trace: NULL pointer array");
    const int n = b->ninst;
    std::vector<tcore::TArgs> A(n);
    std::vector<int64_t> loff(n + 1, 0);
    std::vector<void*> ptrs(4 * (size_t)n, nullptr);
    for (int i = 0; i < n; ++i) {
        if (L[i] < 0 || (L[i] > 0 && (!u[i] || !seeds[i])))
            return berr(b, BEM_ERR_ARG, "bem_batch_trace: bad line count or NULL vector");
        if (int rc = trace_args(b->ctx[i], tp, u[i], &A[i])) return berr(b, rc, bem_last_error(b->ctx[i]));
        loff[i + 1] = loff[i] + L[i];
        ptrs[i] = const_cast<double*>(seeds[i]);
        ptrs[n + i] = K ? K[i] : nullptr;
        ptrs[2 * n + i] = status ? status[i] : nullptr;
        ptrs[3 * n + i] = nsteps ? nsteps[i] : nullptr;
    }
    const int64_t total = loff[n];
    if (total == 0) return BEM_OK;
    if (total > 0x7fffffff) return berr(b, BEM_ERR_ARG, "bem_batch_trace: too many lines");
    if (int rc = enter(b)) return rc;
    cudaStream_t s = b->stream;
    BB_TRY(b, cudaMemcpyAsync(b->d_targs, A.data(), n * sizeof(tcore::TArgs), cudaMemcpyHostToDevice, s));
    BB_TRY(b, cudaMemcpyAsync(b->d_loff, loff.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    BB_TRY(b, cudaMemcpyAsync(b->d_tptr, ptrs.data(), ptrs.size() * sizeof(void*), cudaMemcpyHostToDevice, s));
    BB_TRY(b, cudaMemsetAsync(b->d_lnext, 0, n * sizeof(unsigned long long), s));
    const double* const* d_seeds = (const double* const*)b->d_tptr;
    double* const* d_K = (double* const*)(b->d_tptr + n);
    int32_t* const* d_st = (int32_t* const*)(b->d_tptr + 2 * n);
    int32_t* const* d_ns = (int32_t* const*)(b->d_tptr + 3 * n);
    int rc = BEM_OK;
    // the cluster size for the largest mesh and all lines (the first instance's
    // trace_cluster, if set); a mesh too small to be split is swept by the leader alone,
    // exactly as in its own bem_trace_lines
    int64_t npmax = 0;
    for (int i = 0; i < n; ++i) npmax = std::max(npmax, b->ctx[i]->np);
    const int ncl = tcore::tracer_cluster(npmax, total, b->num_sms, b->ctx[0]->prm.trace_cluster);
    switch (b->g * 2 + (precision == BEM_MIXED ? 1 : 0)) {
#define BT(G, QQ, F32)                                                                                  \
    case G * 2 + F32: {                                                                                 \
        constexpr size_t fsm = tcore::field_smem<F32, QQ>();                                            \
        BB_TRY(b, tcore::allow_smem(k_btrace<F32, QQ>, fsm));                                           \
        const unsigned grid = tcore::lines_grid(k_btrace<F32, QQ>, fsm, b->num_sms, total, ncl);        \
        BB_TRY(b, tcore::launch_lines(k_btrace<F32, QQ>, grid, fsm, s, ncl, (const tcore::TArgs*)b->d_targs, \
                                      (const int64_t*)b->d_loff, n, b->d_lnext, d_seeds, d_K, d_st, d_ns)); \
        break;                                                                                          \
    }
        BT(2, 4, 0) BT(2, 4, 1) BT(3, 9, 0) BT(3, 9, 1) BT(4, 16, 0) BT(4, 16, 1)
#undef BT
        default: rc = berr(b, BEM_ERR_ARG, "batched tracer: far_order must be 2..4");
    }
    if (rc) return rc;
    BB_LAUNCH(b);
    b->cnt.lines += total;
    // the host arrays A, loff, ptrs die on return: wait until the copies have run
    BB_TRY(b, cudaStreamSynchronize(s));
    return leave(b);
}

// ---------------------------------------------------------------- field at points
// Mixed form: every instance's points in chunks of the smallest max_points of the
// contexts; per chunk ONE persistent launch of the regular pairs of all instances
// (items of kTile points x a triangle slice common to all instances, at most four
// slices per instance, written into each context's own far workspace), then each
// instance's deferred FP64 near pass (the kernel of bem_eval_field).  FP64 form: each
// instance's bem_eval_field in turn.
extern "C" int bem_batch_eval_field(bem_batch* b, int32_t precision, const double* const* u,
                                    const int64_t* M, const double* const* pts, double* const* phi,
                                    double* const* E)
{
    if (!b) return BEM_ERR_ARG;
    if (precision != BEM_FP64 && precision != BEM_MIXED)
        return berr(b, BEM_ERR_ARG, "bem_batch_eval_field: precision must be BEM_FP64 or BEM_MIXED");
    if (!u || !M || !pts) return berr(b, BEM_ERR_ARG, "bem_batch_eval_field: NULL array");
    const int n = b->ninst;
    int64_t Mmax = 0, CH = INT64_MAX, npmax = 0;
    for (int i = 0; i < n; ++i) {
        if (M[i] < 0 || (M[i] > 0 && (!u[i] || !pts[i])))
            return berr(b, BEM_ERR_ARG, "bem_batch_eval_field: bad M or NULL pointer");
        Mmax = std::max(Mmax, M[i]);
        CH = std::min<int64_t>(CH, b->ctx[i]->prm.max_points);
        npmax = std::max(npmax, b->ctx[i]->np);
    }
    if (precision == BEM_FP64) {
        for (int i = 0; i < n; ++i) {
            const int rc = bem_eval_field(b->ctx[i], BEM_FP64, u[i], M[i], pts[i], phi ? phi[i] : nullptr,
                                          E ? E[i] : nullptr);
            if (rc) return berr(b, rc, bem_last_error(b->ctx[i]));
        }
        return BEM_OK;
    }
    // a slice length common to all instances: at most four slices of the largest mesh
    const int64_t slice = std::max<int64_t>(kBPC, ((npmax + 3) / 4 + kBPC - 1) / kBPC * kBPC);
    if (int rc = enter(b)) return rc;
    cudaStream_t s = b->stream;
    std::vector<PInst> pi(n);
    std::vector<int64_t> off(n + 1);
    for (int64_t m0 = 0; m0 < Mmax; m0 += CH) {
        off[0] = 0;
        for (int i = 0; i < n; ++i) {
            bem_ctx* c = b->ctx[i];
            PInst& P = pi[i];
            P.M = std::max<int64_t>(0, std::min(CH, M[i] - m0));
            P.pts = P.M > 0 ? pts[i] + 3 * m0 : nullptr;
            P.u = u[i];
            P.hdr32 = c->hdr32;
            P.node32 = c->node32;
            P.part = c->part;
            P.np = c->np;
            P.slice = slice;
            P.splits = (c->np + slice - 1) / slice;
            if ((size_t)P.splits * P.M * 4 > c->part_cap)
                return berr(b, BEM_ERR_CAPACITY, "bem_batch_eval_field: far workspace too small");
            off[i + 1] = off[i] + ((P.M + kTile - 1) / kTile) * P.splits;
        }
        const int64_t total = off[n];
        if (total == 0) continue;
        BB_TRY(b, cudaMemcpyAsync(b->d_pinst, pi.data(), n * sizeof(PInst), cudaMemcpyHostToDevice, s));
        BB_TRY(b, cudaMemcpyAsync(b->d_pitem_off, off.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        BB_TRY(b, cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned long long), s));
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(total, (int64_t)b->num_sms * 4));
        switch (b->g) {
            case 2: k_bfar_pts<4><<<grid, kBT, 0, s>>>(b->d_pinst, n, b->d_pitem_off, total, b->d_queue, b->d_epairs); break;
            case 3: k_bfar_pts<9><<<grid, kBT, 0, s>>>(b->d_pinst, n, b->d_pitem_off, total, b->d_queue, b->d_epairs); break;
            default: k_bfar_pts<16><<<grid, kBT, 0, s>>>(b->d_pinst, n, b->d_pitem_off, total, b->d_queue, b->d_epairs); break;
        }
        BB_LAUNCH(b);
        ++b->cnt.far_launches;
        if (int rc = leave(b)) return rc;
        // the near pass of each instance on the contexts' stream, after the launch above
        for (int i = 0; i < n; ++i) {
            const PInst& P = pi[i];
            if (P.M == 0) continue;
            const int rc = launch_points_near(b->ctx[i], BEM_MIXED, P.M, P.pts, P.u, P.part, (int)P.splits,
                                              phi && phi[i] ? phi[i] + m0 : nullptr,
                                              E && E[i] ? E[i] + 3 * m0 : nullptr);
            if (rc) return berr(b, rc, bem_last_error(b->ctx[i]));
            ++b->cnt.kernel_launches;
        }
        // the next chunk's launch reuses the contexts' far workspaces: order it after
        // the near passes
        if (int rc = enter(b)) return rc;
    }
    // (pi and off are pageable: each copy has taken its bytes before it returns)
    return leave(b);
}

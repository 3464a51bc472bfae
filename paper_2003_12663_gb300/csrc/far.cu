// far.cu -- the regular-pair interaction kernels (Sec. 4, regular pairs by the
// Duffy/Gauss rule).  For every target x_t and every triangle j whose pair with
// x_t is regular (D > eta R), accumulate
//     phi_t += u_j sum_k w_jk / |x_t - y_jk|
//     E_t   += u_j sum_k w_jk (x_t - y_jk) / |x_t - y_jk|^3
// (times 1/(4 pi), applied by the consumers).  Near pairs are skipped here and
// handled in FP64 by the closed form afterwards (the deferred second pass of
// Sec. 4 / Fig. 3).
//
// Layout: one CTA owns a tile of kThreads*TR targets (TR per thread, register
// blocked) and one contiguous slice ("split") of triangles.  Triangles are
// staged through shared memory in chunks of PC: the classification header
// (circumcentre, (eta R)^2), the density u_j and the Q quadrature nodes (y, w),
// each node read by every thread of the CTA for all of its TR targets.  The CTA
// writes one partial (phi, E) per target and split; the consumer adds the
// splits in FP64.
//
// FP32 form: per triangle the Q node contributions are summed in FP32, folded
// into a per-chunk FP32 partial with u_j (masked to 0 for near pairs), and the
// chunk partials are added with Kahan compensation.
#include <algorithm>

#include "bem_internal.cuh"

namespace {

constexpr int kThreads = 128;
constexpr int kTR32 = 4;
constexpr int kTR64 = 2;
constexpr int kTRdf = 2;   // double-FP32, one right-hand side
constexpr int kTRdfN = 2;  // double-FP32, several right-hand sides (registers)
constexpr int kPC32 = 32;
constexpr int kPC64 = 16;

template <int TR, int Q, bool RAW>
__global__ void __launch_bounds__(kThreads)
k_far32(const float4* __restrict__ t32, const double* __restrict__ tpts, int64_t M,
        const float4* __restrict__ hdr, const float4* __restrict__ node,
        const double* __restrict__ u, int64_t np, int64_t per_split, double* __restrict__ part)
{
    constexpr int PC = kPC32;
    __shared__ float4 s_hdr[PC];
    __shared__ float s_u[PC];
    __shared__ float4 s_node[PC * Q];
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * (kThreads * TR);
    const int split = blockIdx.y;
    const int64_t p0 = (int64_t)split * per_split;
    const int64_t p1 = min(np, p0 + per_split);

    float tx[TR], ty[TR], tz[TR];
#pragma unroll
    for (int r = 0; r < TR; ++r) {
        const int64_t t = min(base + r * kThreads + tid, M - 1);
        if (RAW) {
            tx[r] = __double2float_rn(tpts[3 * t]);
            ty[r] = __double2float_rn(tpts[3 * t + 1]);
            tz[r] = __double2float_rn(tpts[3 * t + 2]);
        } else {
            const float4 v = t32[t];
            tx[r] = v.x; ty[r] = v.y; tz[r] = v.z;
        }
    }
    float acc[TR][4], cmp[TR][4];
#pragma unroll
    for (int r = 0; r < TR; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = cmp[r][c] = 0.f;

    for (int64_t c0 = p0; c0 < p1; c0 += PC) {
        const int npc = (int)min((int64_t)PC, p1 - c0);
        __syncthreads();
        for (int k = tid; k < npc; k += kThreads) {
            s_hdr[k] = hdr[c0 + k];
            s_u[k] = __double2float_rn(u[c0 + k]);
        }
        for (int k = tid; k < npc * Q; k += kThreads) s_node[k] = node[c0 * Q + k];
        __syncthreads();
        float cp[TR][4];
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) cp[r][c] = 0.f;
        for (int p = 0; p < npc; ++p) {
            float ps[TR], gx[TR], gy[TR], gz[TR];
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const float4 nd = s_node[p * Q + k];
#pragma unroll
                for (int r = 0; r < TR; ++r) {
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
            const float up = s_u[p];
#pragma unroll
            for (int r = 0; r < TR; ++r) {
                const float m = is_far32(tx[r], ty[r], tz[r], h) ? up : 0.f;
                cp[r][0] = fmaf(m, ps[r], cp[r][0]);
                cp[r][1] = fmaf(m, gx[r], cp[r][1]);
                cp[r][2] = fmaf(m, gy[r], cp[r][2]);
                cp[r][3] = fmaf(m, gz[r], cp[r][3]);
            }
        }
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) {  // Kahan: acc + cmp carries the exact running sum
                const float y = cp[r][c] - cmp[r][c];
                const float t = acc[r][c] + y;
                cmp[r][c] = (t - acc[r][c]) - y;
                acc[r][c] = t;
            }
    }
#pragma unroll
    for (int r = 0; r < TR; ++r) {
        const int64_t t = base + r * kThreads + tid;
        if (t < M) {
            double* o = part + ((int64_t)split * M + t) * 4;
            o[0] = (double)acc[r][0] - (double)cmp[r][0];
            o[1] = (double)acc[r][1] - (double)cmp[r][1];
            o[2] = (double)acc[r][2] - (double)cmp[r][2];
            o[3] = (double)acc[r][3] - (double)cmp[r][3];
        }
    }
}

// ---------------------------------------------------------------- packed FP32
// The same regular-pair sums with Blackwell's paired FP32 instructions
// (add/mul/fma on float2): every thread holds 2*TP targets as TP pairs, so one
// instruction advances two pair-ops and the FP32 units, not instruction issue,
// set the pace.  The node stream arrives with sigma folded into the weights
// (k_prescale) and already duplicated into pairs (-y, -y, w) in shared memory.
// Before each chunk of PC triangles the CTA compares the bounding sphere of its
// targets with the chunk's precomputed sphere (circumcentres + eta R, with a
// rounding margin): if every pair is certainly regular, the chunk runs as a flat
// node stream without any per-triangle classification ("fast"); otherwise each
// triangle's sums are masked per target by is_far32, exactly like k_far32.
__global__ void k_prescale(int64_t n, int Q, const float4* __restrict__ node,
                           const double* __restrict__ u, float4* __restrict__ qnode)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 v = node[i];
    v.w = v.w * __double2float_rn(u[i / Q]);
    qnode[i] = v;
}

template <int TP, int Q, bool RAW>
__global__ void __launch_bounds__(kThreads, TP == 3 ? 3 : 1)
k_far32p(const float4* __restrict__ t32, const double* __restrict__ tpts, int64_t M,
         const float4* __restrict__ hdr, const float4* __restrict__ qnode,
         const float4* __restrict__ chunk_sph, int64_t np, int64_t per_split,
         double* __restrict__ part, const int32_t* __restrict__ phi_kind,
         unsigned long long* __restrict__ chunk_stats)
{
    constexpr int PC = kPC32;
    constexpr int TR = 2 * TP;
    __shared__ float4 s_hdr[PC];
    __shared__ float4 s_n2[PC * Q][2];   // (-x,-x,-y,-y), (-z,-z,w,w)
    __shared__ float s_box[6][kThreads / 32];
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * (kThreads * TR);
    const int split = blockIdx.y;
    const int64_t p0 = (int64_t)split * per_split;
    const int64_t p1 = min(np, p0 + per_split);

    float2 tx[TP], ty[TP], tz[TP];
    float bmin[3] = {3e38f, 3e38f, 3e38f}, bmax[3] = {-3e38f, -3e38f, -3e38f};
#pragma unroll
    for (int q = 0; q < TP; ++q) {
        float v[2][3];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t t = min(base + (2 * q + h) * kThreads + tid, M - 1);
            if (RAW) {
                v[h][0] = __double2float_rn(tpts[3 * t]);
                v[h][1] = __double2float_rn(tpts[3 * t + 1]);
                v[h][2] = __double2float_rn(tpts[3 * t + 2]);
            } else {
                const float4 a = t32[t];
                v[h][0] = a.x; v[h][1] = a.y; v[h][2] = a.z;
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                bmin[c] = fminf(bmin[c], v[h][c]);
                bmax[c] = fmaxf(bmax[c], v[h][c]);
            }
        }
        tx[q] = make_float2(v[0][0], v[1][0]);
        ty[q] = make_float2(v[0][1], v[1][1]);
        tz[q] = make_float2(v[0][2], v[1][2]);
    }
    // bounding box of the CTA's targets -> centre and radius (uniform)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            bmin[c] = fminf(bmin[c], __shfl_xor_sync(0xffffffffu, bmin[c], o));
            bmax[c] = fmaxf(bmax[c], __shfl_xor_sync(0xffffffffu, bmax[c], o));
        }
    if ((tid & 31) == 0)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            s_box[c][tid >> 5] = bmin[c];
            s_box[3 + c][tid >> 5] = bmax[c];
        }
    __syncthreads();
    float tc[3], tr = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        float lo = s_box[c][0], hi = s_box[3 + c][0];
#pragma unroll
        for (int w = 1; w < kThreads / 32; ++w) {
            lo = fminf(lo, s_box[c][w]);
            hi = fmaxf(hi, s_box[3 + c][w]);
        }
        tc[c] = 0.5f * (lo + hi);
        tr += (hi - lo) * (hi - lo);
    }
    tr = 0.5f * sqrtf(tr) * 1.0001f + 1e-6f;
    // a tile of conductor rows only needs phi (their row equation is phi = V0)
    bool mine = phi_kind != nullptr;
    if (phi_kind)
#pragma unroll
        for (int q = 0; q < TP; ++q)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t t = base + (2 * q + h) * kThreads + tid;
                if (t < M) mine = mine && phi_kind[t] == BEM_CONDUCTOR;
            }
    const bool phi_only = __syncthreads_and(mine) != 0;

    float2 acc[TP][4], cmp[TP][4];
#pragma unroll
    for (int q = 0; q < TP; ++q)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[q][c] = cmp[q][c] = make_float2(0.f, 0.f);
    const float2 eps2 = make_float2(1e-20f, 1e-20f);
    unsigned n_chunks = 0, n_fast = 0;  // chunk statistics (thread 0)

    for (int64_t c0 = p0; c0 < p1; c0 += PC) {
        const int npc = (int)min((int64_t)PC, p1 - c0);
        __syncthreads();
        for (int k = tid; k < npc; k += kThreads) s_hdr[k] = hdr[c0 + k];
        for (int k = tid; k < npc * Q; k += kThreads) {
            const float4 v = qnode[c0 * Q + k];
            s_n2[k][0] = make_float4(-v.x, -v.x, -v.y, -v.y);
            s_n2[k][1] = make_float4(-v.z, -v.z, v.w, v.w);
        }
        __syncthreads();
        const float4 cs = chunk_sph[c0 / PC];
        const float ddx = cs.x - tc[0], ddy = cs.y - tc[1], ddz = cs.z - tc[2];
        const bool fast = sqrtf(ddx * ddx + ddy * ddy + ddz * ddz) > tr + cs.w;
        ++n_chunks;
        n_fast += fast ? 1u : 0u;
        float2 cp[TP][4];
#pragma unroll
        for (int q = 0; q < TP; ++q)
#pragma unroll
            for (int c = 0; c < 4; ++c) cp[q][c] = make_float2(0.f, 0.f);
        if (fast && phi_only) {
            for (int p = 0; p < npc; ++p) {
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    const float4 a = s_n2[p * Q + k][0], b = s_n2[p * Q + k][1];
                    const float2 mx = make_float2(a.x, a.y), my = make_float2(a.z, a.w);
                    const float2 mz = make_float2(b.x, b.y), w2 = make_float2(b.z, b.w);
#pragma unroll
                    for (int q = 0; q < TP; ++q) {
                        const float2 dx = __fadd2_rn(tx[q], mx), dy = __fadd2_rn(ty[q], my),
                                     dz = __fadd2_rn(tz[q], mz);
                        const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, eps2)));
                        const float2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
                        cp[q][0] = __ffma2_rn(w2, ri, cp[q][0]);
                    }
                }
            }
        } else if (fast) {
            for (int p = 0; p < npc; ++p) {
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    const float4 a = s_n2[p * Q + k][0], b = s_n2[p * Q + k][1];
                    const float2 mx = make_float2(a.x, a.y), my = make_float2(a.z, a.w);
                    const float2 mz = make_float2(b.x, b.y), w2 = make_float2(b.z, b.w);
#pragma unroll
                    for (int q = 0; q < TP; ++q) {
                        const float2 dx = __fadd2_rn(tx[q], mx), dy = __fadd2_rn(ty[q], my),
                                     dz = __fadd2_rn(tz[q], mz);
                        const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, eps2)));
                        const float2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
                        const float2 t = __fmul2_rn(w2, ri);
                        const float2 t3 = __fmul2_rn(t, __fmul2_rn(ri, ri));
                        cp[q][0] = __fadd2_rn(cp[q][0], t);
                        cp[q][1] = __ffma2_rn(t3, dx, cp[q][1]);
                        cp[q][2] = __ffma2_rn(t3, dy, cp[q][2]);
                        cp[q][3] = __ffma2_rn(t3, dz, cp[q][3]);
                    }
                }
            }
        } else if (phi_only) {
            for (int p = 0; p < npc; ++p) {
                float2 ps[TP];
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    const float4 a = s_n2[p * Q + k][0], b = s_n2[p * Q + k][1];
                    const float2 mx = make_float2(a.x, a.y), my = make_float2(a.z, a.w);
                    const float2 mz = make_float2(b.x, b.y), w2 = make_float2(b.z, b.w);
#pragma unroll
                    for (int q = 0; q < TP; ++q) {
                        const float2 dx = __fadd2_rn(tx[q], mx), dy = __fadd2_rn(ty[q], my),
                                     dz = __fadd2_rn(tz[q], mz);
                        const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, eps2)));
                        const float2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
                        ps[q] = k == 0 ? __fmul2_rn(w2, ri) : __ffma2_rn(w2, ri, ps[q]);
                    }
                }
                const float4 h = s_hdr[p];
#pragma unroll
                for (int q = 0; q < TP; ++q) {
                    const bool f0 = is_far32(tx[q].x, ty[q].x, tz[q].x, h);
                    const bool f1 = is_far32(tx[q].y, ty[q].y, tz[q].y, h);
                    cp[q][0] = __fadd2_rn(cp[q][0], make_float2(f0 ? ps[q].x : 0.f, f1 ? ps[q].y : 0.f));
                }
            }
        } else {
            for (int p = 0; p < npc; ++p) {
                float2 ps[TP], gx[TP], gy[TP], gz[TP];
#pragma unroll
                for (int k = 0; k < Q; ++k) {
                    const float4 a = s_n2[p * Q + k][0], b = s_n2[p * Q + k][1];
                    const float2 mx = make_float2(a.x, a.y), my = make_float2(a.z, a.w);
                    const float2 mz = make_float2(b.x, b.y), w2 = make_float2(b.z, b.w);
#pragma unroll
                    for (int q = 0; q < TP; ++q) {
                        const float2 dx = __fadd2_rn(tx[q], mx), dy = __fadd2_rn(ty[q], my),
                                     dz = __fadd2_rn(tz[q], mz);
                        const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __ffma2_rn(dz, dz, eps2)));
                        const float2 ri = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
                        const float2 t = __fmul2_rn(w2, ri);
                        const float2 t3 = __fmul2_rn(t, __fmul2_rn(ri, ri));
                        if (k == 0) {
                            ps[q] = t;
                            gx[q] = __fmul2_rn(t3, dx); gy[q] = __fmul2_rn(t3, dy); gz[q] = __fmul2_rn(t3, dz);
                        } else {
                            ps[q] = __fadd2_rn(ps[q], t);
                            gx[q] = __ffma2_rn(t3, dx, gx[q]);
                            gy[q] = __ffma2_rn(t3, dy, gy[q]);
                            gz[q] = __ffma2_rn(t3, dz, gz[q]);
                        }
                    }
                }
                const float4 h = s_hdr[p];
#pragma unroll
                for (int q = 0; q < TP; ++q) {
                    const bool f0 = is_far32(tx[q].x, ty[q].x, tz[q].x, h);
                    const bool f1 = is_far32(tx[q].y, ty[q].y, tz[q].y, h);
                    cp[q][0] = __fadd2_rn(cp[q][0], make_float2(f0 ? ps[q].x : 0.f, f1 ? ps[q].y : 0.f));
                    cp[q][1] = __fadd2_rn(cp[q][1], make_float2(f0 ? gx[q].x : 0.f, f1 ? gx[q].y : 0.f));
                    cp[q][2] = __fadd2_rn(cp[q][2], make_float2(f0 ? gy[q].x : 0.f, f1 ? gy[q].y : 0.f));
                    cp[q][3] = __fadd2_rn(cp[q][3], make_float2(f0 ? gz[q].x : 0.f, f1 ? gz[q].y : 0.f));
                }
            }
        }
#pragma unroll
        for (int q = 0; q < TP; ++q)
#pragma unroll
            for (int c = 0; c < 4; ++c) {  // Kahan: acc + cmp carries the running sum
                const float2 y = __fadd2_rn(cp[q][c], make_float2(-cmp[q][c].x, -cmp[q][c].y));
                const float2 t = __fadd2_rn(acc[q][c], y);
                const float2 dd = __fadd2_rn(t, make_float2(-acc[q][c].x, -acc[q][c].y));
                cmp[q][c] = __fadd2_rn(dd, make_float2(-y.x, -y.y));
                acc[q][c] = t;
            }
    }
#pragma unroll
    for (int q = 0; q < TP; ++q)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t t = base + (2 * q + h) * kThreads + tid;
            if (t < M) {
                double* o = part + ((int64_t)split * M + t) * 4;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float a = h ? acc[q][c].y : acc[q][c].x, m = h ? cmp[q][c].y : cmp[q][c].x;
                    o[c] = (double)a - (double)m;
                }
            }
        }
    if (tid == 0 && chunk_stats) {
        atomicAdd(chunk_stats, (unsigned long long)n_chunks);
        atomicAdd(chunk_stats + 1, (unsigned long long)n_fast);
    }
}

template <int TR, int Q, bool RAW>
__global__ void __launch_bounds__(kThreads)
k_far64(const double4* __restrict__ t64, const double* __restrict__ tpts, int64_t M,
        const double4* __restrict__ hdr, const double4* __restrict__ node,
        const double* __restrict__ u, int64_t np, int64_t per_split, double* __restrict__ part)
{
    constexpr int PC = kPC64;
    __shared__ double4 s_hdr[PC];
    __shared__ double s_u[PC];
    __shared__ double4 s_node[PC * Q];
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * (kThreads * TR);
    const int split = blockIdx.y;
    const int64_t p0 = (int64_t)split * per_split;
    const int64_t p1 = min(np, p0 + per_split);

    double tx[TR], ty[TR], tz[TR];
#pragma unroll
    for (int r = 0; r < TR; ++r) {
        const int64_t t = min(base + r * kThreads + tid, M - 1);
        if (RAW) {
            tx[r] = tpts[3 * t]; ty[r] = tpts[3 * t + 1]; tz[r] = tpts[3 * t + 2];
        } else {
            const double4 v = t64[t];
            tx[r] = v.x; ty[r] = v.y; tz[r] = v.z;
        }
    }
    double acc[TR][4];
#pragma unroll
    for (int r = 0; r < TR; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;

    for (int64_t c0 = p0; c0 < p1; c0 += PC) {
        const int npc = (int)min((int64_t)PC, p1 - c0);
        __syncthreads();
        for (int k = tid; k < npc; k += kThreads) {
            s_hdr[k] = hdr[c0 + k];
            s_u[k] = u[c0 + k];
        }
        for (int k = tid; k < npc * Q; k += kThreads) s_node[k] = node[c0 * Q + k];
        __syncthreads();
        for (int p = 0; p < npc; ++p) {
            double ps[TR], gx[TR], gy[TR], gz[TR];
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const double4 nd = s_node[p * Q + k];
#pragma unroll
                for (int r = 0; r < TR; ++r) {
                    const double dx = tx[r] - nd.x, dy = ty[r] - nd.y, dz = tz[r] - nd.z;
                    const double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, 1e-200)));
                    const double ri = rsqrt(r2);
                    const double t = nd.w * ri;
                    const double t3 = t * (ri * ri);
                    if (k == 0) {
                        ps[r] = t;
                        gx[r] = t3 * dx; gy[r] = t3 * dy; gz[r] = t3 * dz;
                    } else {
                        ps[r] += t;
                        gx[r] = fma(t3, dx, gx[r]);
                        gy[r] = fma(t3, dy, gy[r]);
                        gz[r] = fma(t3, dz, gz[r]);
                    }
                }
            }
            const double4 h = s_hdr[p];
            const double up = s_u[p];
#pragma unroll
            for (int r = 0; r < TR; ++r) {
                const double m = is_far64(tx[r], ty[r], tz[r], h) ? up : 0.0;
                acc[r][0] = fma(m, ps[r], acc[r][0]);
                acc[r][1] = fma(m, gx[r], acc[r][1]);
                acc[r][2] = fma(m, gy[r], acc[r][2]);
                acc[r][3] = fma(m, gz[r], acc[r][3]);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < TR; ++r) {
        const int64_t t = base + r * kThreads + tid;
        if (t < M) {
            double* o = part + ((int64_t)split * M + t) * 4;
            o[0] = acc[r][0]; o[1] = acc[r][1]; o[2] = acc[r][2]; o[3] = acc[r][3];
        }
    }
}

// ---------------------------------------------------------------- double-FP32
// A value is the unevaluated sum hi + lo of two floats (|lo| <= ulp(hi)/2).  The
// operations are the error-free transformations of Knuth (two-sum) and Dekker
// (two-product, here with an FMA), written with explicit-rounding intrinsics so
// that the compiler cannot fuse or reorder them.
struct df32 {
    float hi, lo;
};

__device__ __forceinline__ df32 quick_two_sum(float a, float b)  // needs |a| >= |b|
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df32 df_add(df32 a, df32 b)
{
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    return quick_two_sum(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df32 df_neg(df32 a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ df32 df_mul(df32 a, df32 b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    return quick_two_sum(p, e);
}

__device__ __forceinline__ df32 df_sqr(df32 a)
{
    const float p = __fmul_rn(a.hi, a.hi);
    const float e = __fmaf_rn(__fadd_rn(a.hi, a.hi), a.lo, __fmaf_rn(a.hi, a.hi, -p));
    return quick_two_sum(p, e);
}

// 1/sqrt(x): the FP32 estimate y, then one Newton step y + y (1 - x y^2) / 2 in
// double-FP32 (the error goes from ~2^-22 to ~2^-44).
__device__ __forceinline__ df32 df_rsqrt(df32 x)
{
    const float y = rsqrtf(x.hi);
    const df32 yy = {__fmul_rn(y, y), __fmaf_rn(y, y, -__fmul_rn(y, y))};
    const df32 t = df_mul(x, yy);
    const float d = __fsub_rn(__fsub_rn(1.0f, t.hi), t.lo);
    return quick_two_sum(y, __fmul_rn(__fmul_rn(y, d), 0.5f));
}

__device__ __forceinline__ df32 df_from(double v)
{
    const float h = __double2float_rn(v);
    return {h, __double2float_rn(v - (double)h)};
}

// Regular pairs in double-FP32, centroid targets only (the refinement residual).
// Near pairs are masked with the FP32 classification, exactly as in k_far32; the
// consumer adds per near pair the value that turns the result into the FP64
// classification's (see k_near_values).  NR right-hand sides (densities
// u + r * ustride) share one pass over the nodes: the node sums of a pair do not
// depend on the density; each right-hand side's arithmetic is that of NR = 1.
template <int TR, int Q, int NR>
__global__ void __launch_bounds__(kThreads)
k_far_df(const float4* __restrict__ t32, const float4* __restrict__ t32lo, int64_t M,
         const float4* __restrict__ hdr, const float4* __restrict__ node,
         const float4* __restrict__ node_lo, const double* __restrict__ u, int64_t ustride,
         int64_t np, int64_t per_split, double* __restrict__ part)
{
    constexpr int PC = 16;
    __shared__ float4 s_hdr[PC];
    __shared__ float2 s_u[NR][PC];
    __shared__ float4 s_node[PC * Q];
    __shared__ float4 s_nlo[PC * Q];
    const int tid = threadIdx.x;
    const int64_t base = (int64_t)blockIdx.x * (kThreads * TR);
    const int split = blockIdx.y;
    const int64_t p0 = (int64_t)split * per_split;
    const int64_t p1 = min(np, p0 + per_split);

    df32 tx[TR], ty[TR], tz[TR];
    float fx[TR], fy[TR], fz[TR];  // FP32 targets of the classification
#pragma unroll
    for (int r = 0; r < TR; ++r) {
        const int64_t t = min(base + r * kThreads + tid, M - 1);
        const float4 h = t32[t], l = t32lo[t];
        tx[r] = {h.x, l.x}; ty[r] = {h.y, l.y}; tz[r] = {h.z, l.z};
        fx[r] = h.x; fy[r] = h.y; fz[r] = h.z;
    }
    df32 acc[NR][TR][4];
#pragma unroll
    for (int q = 0; q < NR; ++q)
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[q][r][c] = {0.f, 0.f};

    for (int64_t c0 = p0; c0 < p1; c0 += PC) {
        const int npc = (int)min((int64_t)PC, p1 - c0);
        __syncthreads();
        for (int k = tid; k < npc; k += kThreads) {
            s_hdr[k] = hdr[c0 + k];
#pragma unroll
            for (int q = 0; q < NR; ++q) {
                const df32 v = df_from(u[q * ustride + c0 + k]);
                s_u[q][k] = make_float2(v.hi, v.lo);
            }
        }
        for (int k = tid; k < npc * Q; k += kThreads) {
            s_node[k] = node[c0 * Q + k];
            s_nlo[k] = node_lo[c0 * Q + k];
        }
        __syncthreads();
        for (int p = 0; p < npc; ++p) {
            df32 ps[TR], gx[TR], gy[TR], gz[TR];
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const float4 nh = s_node[p * Q + k], nl = s_nlo[p * Q + k];
                const df32 w = {nh.w, nl.w};
#pragma unroll
                for (int r = 0; r < TR; ++r) {
                    const df32 dx = df_add(tx[r], df_neg({nh.x, nl.x}));
                    const df32 dy = df_add(ty[r], df_neg({nh.y, nl.y}));
                    const df32 dz = df_add(tz[r], df_neg({nh.z, nl.z}));
                    df32 r2 = df_add(df_add(df_sqr(dx), df_sqr(dy)), df_sqr(dz));
                    r2.hi = fmaxf(r2.hi, 1e-20f);
                    const df32 ri = df_rsqrt(r2);
                    const df32 t = df_mul(w, ri);
                    const df32 t3 = df_mul(t, df_sqr(ri));
                    if (k == 0) {
                        ps[r] = t;
                        gx[r] = df_mul(t3, dx); gy[r] = df_mul(t3, dy); gz[r] = df_mul(t3, dz);
                    } else {
                        ps[r] = df_add(ps[r], t);
                        gx[r] = df_add(gx[r], df_mul(t3, dx));
                        gy[r] = df_add(gy[r], df_mul(t3, dy));
                        gz[r] = df_add(gz[r], df_mul(t3, dz));
                    }
                }
            }
            const float4 h = s_hdr[p];
#pragma unroll
            for (int r = 0; r < TR; ++r) {
                const bool far = is_far32(fx[r], fy[r], fz[r], h);
#pragma unroll
                for (int q = 0; q < NR; ++q) {
                    const float2 up = s_u[q][p];
                    const df32 m = far ? df32{up.x, up.y} : df32{0.f, 0.f};
                    acc[q][r][0] = df_add(acc[q][r][0], df_mul(m, ps[r]));
                    acc[q][r][1] = df_add(acc[q][r][1], df_mul(m, gx[r]));
                    acc[q][r][2] = df_add(acc[q][r][2], df_mul(m, gy[r]));
                    acc[q][r][3] = df_add(acc[q][r][3], df_mul(m, gz[r]));
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < NR; ++q)
#pragma unroll
        for (int r = 0; r < TR; ++r) {
            const int64_t t = base + r * kThreads + tid;
            if (t < M) {
                double* o = part + (((int64_t)q * gridDim.y + split) * M + t) * 4;
#pragma unroll
                for (int c = 0; c < 4; ++c) o[c] = (double)acc[q][r][c].hi + (double)acc[q][r][c].lo;
            }
        }
}

template <int Q>
int launch_q(bem_ctx* ctx, int precision, const FarTargets& T, const double* u, int splits,
             double* part)
{
    const int64_t np = ctx->np;
    // slices start on whole 32-triangle chunks (the chunk spheres of k_far32p)
    const int64_t per_split = ((np + splits - 1) / splits + kPC32 - 1) / kPC32 * kPC32;
    const bool raw = (T.tpts != nullptr);
    if (ctx->p1 && (precision == kPrecDF || (precision == BEM_MIXED && ctx->far32_tp < 2)))
        return set_err(ctx, BEM_ERR_ARG, "curved triangles: packed FP32 or FP64 regular pairs only");
    if (precision == BEM_MIXED && ctx->far32_tp > 1) {
        if (!ctx->p1) {  // a curved-triangle context folds its density itself
            const int64_t n = np * Q;
            k_prescale<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(n, Q, ctx->node32, u, ctx->qnode);
            BEM_LAUNCH_CHECK(ctx);
        }
        const int tr = 2 * ctx->far32_tp;
        dim3 grid((unsigned)((T.M + kThreads * tr - 1) / (kThreads * tr)), (unsigned)splits);
#define FAR32P(TP)                                                                                     \
    if (raw)                                                                                           \
        k_far32p<TP, Q, true><<<grid, kThreads, 0, ctx->stream>>>(                                     \
            nullptr, T.tpts, T.M, ctx->hdr32, ctx->qnode, ctx->chunk_sph, np, per_split, part, nullptr, \
            ctx->d_near_count + 2);                                                                    \
    else                                                                                               \
        k_far32p<TP, Q, false><<<grid, kThreads, 0, ctx->stream>>>(                                    \
            T.t32, nullptr, T.M, ctx->hdr32, ctx->qnode, ctx->chunk_sph, np, per_split, part, T.phi_kind, \
            ctx->d_near_count + 2)
        if (ctx->far32_tp == 4) {
            FAR32P(4);
        } else if (ctx->far32_tp == 3) {
            FAR32P(3);
        } else {
            FAR32P(2);
        }
#undef FAR32P
    } else if (precision == kPrecDF) {
        if (raw || !T.t32lo) return set_err(ctx, BEM_ERR_ARG, "double-FP32 pass needs centroid targets");
        dim3 grid((unsigned)((T.M + kThreads * kTRdf - 1) / (kThreads * kTRdf)), (unsigned)splits);
        k_far_df<kTRdf, Q, 1><<<grid, kThreads, 0, ctx->stream>>>(
            T.t32, T.t32lo, T.M, ctx->hdr32, ctx->node32, ctx->node_lo32, u, 0, np, per_split, part);
    } else if (precision == BEM_MIXED) {
        dim3 grid((unsigned)((T.M + kThreads * kTR32 - 1) / (kThreads * kTR32)), (unsigned)splits);
        if (raw)
            k_far32<kTR32, Q, true><<<grid, kThreads, 0, ctx->stream>>>(
                nullptr, T.tpts, T.M, ctx->hdr32, ctx->node32, u, np, per_split, part);
        else
            k_far32<kTR32, Q, false><<<grid, kThreads, 0, ctx->stream>>>(
                T.t32, nullptr, T.M, ctx->hdr32, ctx->node32, u, np, per_split, part);
    } else {
        // a curved-triangle context passes its folded nodes with a unit density
        const double4* nodes = ctx->p1 ? ctx->qnode64 : ctx->node64;
        dim3 grid((unsigned)((T.M + kThreads * kTR64 - 1) / (kThreads * kTR64)), (unsigned)splits);
        if (raw)
            k_far64<kTR64, Q, true><<<grid, kThreads, 0, ctx->stream>>>(
                nullptr, T.tpts, T.M, ctx->hdr64, nodes, u, np, per_split, part);
        else
            k_far64<kTR64, Q, false><<<grid, kThreads, 0, ctx->stream>>>(
                T.t64, nullptr, T.M, ctx->hdr64, nodes, u, np, per_split, part);
    }
    BEM_LAUNCH_CHECK(ctx);
    return BEM_OK;
}

// double-FP32 pass of nrhs (2..4) right-hand sides in one launch (g = 2..4)
template <int Q>
int launch_df_multi(bem_ctx* ctx, const FarTargets& T, const double* u, int nrhs, int64_t ustride,
                    int splits, double* part)
{
    if (T.tpts || !T.t32lo) return set_err(ctx, BEM_ERR_ARG, "double-FP32 pass needs centroid targets");
    const int64_t np = ctx->np;
    const int64_t per_split = ((np + splits - 1) / splits + kPC32 - 1) / kPC32 * kPC32;
    dim3 grid((unsigned)((T.M + kThreads * kTRdfN - 1) / (kThreads * kTRdfN)), (unsigned)splits);
#define DFM(NR)                                                                                       \
    k_far_df<kTRdfN, Q, NR><<<grid, kThreads, 0, ctx->stream>>>(T.t32, T.t32lo, T.M, ctx->hdr32,         \
                                                               ctx->node32, ctx->node_lo32, u, ustride, \
                                                               np, per_split, part)
    switch (nrhs) {
        case 2: DFM(2); break;
        case 3: DFM(3); break;
        case 4: DFM(4); break;
        default: return set_err(ctx, BEM_ERR_ARG, "double-FP32 pass: nrhs %d", nrhs);
    }
#undef DFM
    BEM_LAUNCH_CHECK(ctx);
    return BEM_OK;
}

}  // namespace

// Number of triangle slices for M targets: enough CTAs to give every SM about
// four, but no slice shorter than two staging chunks.
int far_splits(const bem_ctx* ctx, int precision, int64_t M)
{
    const int tr = precision == BEM_MIXED ? (ctx->far32_tp > 1 ? 2 * ctx->far32_tp : kTR32)
                                          : (precision == kPrecDF ? kTRdf : kTR64);
    const int pc = precision == BEM_MIXED ? kPC32 : kPC64;
    const int64_t tiles = (M + kThreads * tr - 1) / (kThreads * tr);
    const int64_t slots = (int64_t)std::max(ctx->num_sms, 1) * (precision == BEM_MIXED ? ctx->far_slots : 4);
    int64_t s = tiles >= slots ? 1 : slots / std::max<int64_t>(tiles, 1);
    s = std::min<int64_t>(s, std::max<int64_t>(1, ctx->np / (2 * pc)));
    s = std::max<int64_t>(1, std::min<int64_t>(s, 64));
    return (int)s;
}

int64_t far_phi_tile_targets(const bem_ctx* ctx)
{
    if (ctx->far32_tp <= 1) return 0;
    const int64_t tile = (int64_t)kThreads * 2 * ctx->far32_tp, np = ctx->np;
    int64_t n = 0;
    for (int64_t t0 = 0; t0 < np; t0 += tile) {
        const int64_t t1 = std::min(np, t0 + tile);
        bool all = true;
        for (int64_t t = t0; t < t1 && all; ++t)
            all = ctx->regions[ctx->h_region[t]].kind == BEM_CONDUCTOR;
        if (all) n += t1 - t0;
    }
    return n;
}

int launch_far(bem_ctx* ctx, int precision, const FarTargets& T, const double* u, int nrhs,
               int64_t ustride, int splits, double* part)
{
    if (T.M <= 0) return BEM_OK;
    const int pi = precision;  // BEM_FP64, BEM_MIXED or kPrecDF
    if (precision == kPrecDF && nrhs > 1 && ctx->g >= 2 && ctx->g <= 4) {
        // all right-hand sides in one pass; part holds [nrhs][splits][M][4]
        ctx->cnt.far_launches[pi] += 1;
        ctx->cnt.pairs[pi] += nrhs * T.M * ctx->np;
        if (T.tpts == nullptr) ctx->cnt.near_pairs[pi] += nrhs * ctx->nnz_prec[pi];
        timing_begin(ctx, pi);
        int rc;
        switch (ctx->g) {
            case 2: rc = launch_df_multi<4>(ctx, T, u, nrhs, ustride, splits, part); break;
            case 3: rc = launch_df_multi<9>(ctx, T, u, nrhs, ustride, splits, part); break;
            default: rc = launch_df_multi<16>(ctx, T, u, nrhs, ustride, splits, part); break;
        }
        timing_end(ctx);
        return rc;
    }
    for (int r = 0; r < nrhs; ++r) {
        const double* ur = u + r * ustride;
        double* pr = part + (size_t)r * splits * T.M * 4;
        int rc;
        ctx->cnt.far_launches[pi] += 1;
        ctx->cnt.pairs[pi] += T.M * ctx->np;
        if (T.tpts == nullptr) ctx->cnt.near_pairs[pi] += ctx->nnz_prec[pi];  // centroid targets
        if (precision == BEM_MIXED && T.phi_kind && T.tpts == nullptr)
            ctx->cnt.phi_pairs[pi] += ctx->phi_tile_targets * ctx->np;
        timing_begin(ctx, pi);
        switch (ctx->g) {
            case 1: rc = launch_q<1>(ctx, precision, T, ur, splits, pr); break;
            case 2: rc = launch_q<4>(ctx, precision, T, ur, splits, pr); break;
            case 3: rc = launch_q<9>(ctx, precision, T, ur, splits, pr); break;
            case 4: rc = launch_q<16>(ctx, precision, T, ur, splits, pr); break;
            case 5: rc = launch_q<25>(ctx, precision, T, ur, splits, pr); break;
            case 6: rc = launch_q<36>(ctx, precision, T, ur, splits, pr); break;
            default: return set_err(ctx, BEM_ERR_ARG, "far_order %d not compiled", ctx->g);
        }
        timing_end(ctx);
        if (rc) return rc;
    }
    return BEM_OK;
}

// field.cu -- everything after the regular-pair pass: the deferred near pairs in
// FP64 (Sec. 4, Fig. 3), the row equations of Eqs. Final1-Final4 (matrix-free
// matvec and dense rows), the surface field and the field at arbitrary points.
#include "bem_internal.cuh"

namespace {

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One warp per collocation row i: add the far partials over the splits and the
// near pairs of the row (closed form, FP64), giving phi(c_i) and E_PV(c_i); then
// the row equation.  mode 0: matvec (y, neutrality terms); mode 1: surface
// field E+ = E_PV + u_i n_i / 2.
__global__ void k_rows(int64_t np, int splits, const double* __restrict__ part,
                       const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                       const double4* __restrict__ val, const uint8_t* __restrict__ flag,
                       uint8_t bit, const double* __restrict__ x, const double* __restrict__ geo,
                       const int32_t* __restrict__ kind, const int32_t* __restrict__ aux,
                       const double* __restrict__ ra, const double* __restrict__ rb,
                       const double* __restrict__ rw, const double* __restrict__ rs, int mode,
                       double* __restrict__ y, double* __restrict__ neut, double* __restrict__ field)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= np) return;
    double p = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
    for (int s = lane; s < splits; s += 32) {
        const double* q = part + ((int64_t)s * np + i) * 4;
        p += q[0]; ex += q[1]; ey += q[2]; ez += q[3];
    }
    p *= kInv4Pi; ex *= kInv4Pi; ey *= kInv4Pi; ez *= kInv4Pi;
    for (int64_t k = ptr[i] + lane; k < ptr[i + 1]; k += 32) {
        if (flag[k] & bit) {
            const double uj = x[col[k]];
            const double4 v = val[k];
            p = fma(uj, v.x, p);
            ex = fma(uj, v.y, ex);
            ey = fma(uj, v.z, ey);
            ez = fma(uj, v.w, ez);
        }
    }
    p = warp_sum(p); ex = warp_sum(ex); ey = warp_sum(ey); ez = warp_sum(ez);
    if (lane != 0) return;
    const double* gp = geo + GEO_STRIDE * i;
    const double nx = gp[GEO_N], ny = gp[GEO_N + 1], nz = gp[GEO_N + 2];
    const double en = ex * nx + ey * ny + ez * nz;  // (K'u)_i, Eq. ADL
    if (field) {
        double* f = field + 4 * i;
        f[0] = p; f[1] = ex; f[2] = ey; f[3] = ez;
    }
    if (mode == 1) {
        const double h = 0.5 * x[i];
        double* f = y + 3 * i;
        f[0] = ex + h * nx; f[1] = ey + h * ny; f[2] = ez + h * nz;
        return;
    }
    const int kd = kind[i];
    double yi;
    if (kd == BEM_CONDUCTOR) {
        yi = p;                                   // Eq. Final1
    } else if (kd == BEM_FLOATING) {
        yi = p - x[np + aux[i]];                  // Eq. Final2
    } else {
        yi = ra[i] * x[i] + rb[i] * en;           // Eq. Final3
    }
    y[i] = yi;
    // Eq. Final4 summand (Eq. sheets for the rows of a sheet: rs_i != 0)
    neut[i] = (kd == BEM_FLOATING) ? rw[i] * (0.5 * x[i] + en) + rs[i] * x[i] : 0.0;
}

// One block per floating body: y[N+f] = sum of its rows' neutrality terms, in a
// fixed order (deterministic).  A body has thousands of rows: 1024 threads keep the
// gathers in flight.
constexpr int kNeutThreads = 1024;
__global__ void k_neutrality(int64_t np, const int32_t* __restrict__ rows,
                             const int32_t* __restrict__ off, const double* __restrict__ neut,
                             double* __restrict__ y)
{
    __shared__ double sh[kNeutThreads];
    const int f = blockIdx.x;
    double s = 0.0;
#pragma unroll 4
    for (int k = off[f] + threadIdx.x; k < off[f + 1]; k += kNeutThreads) s += neut[rows[k]];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) y[np + f] = sh[0];
}

__global__ void k_rhs(int64_t np, int64_t nunk, int nregions, const int32_t* __restrict__ kind,
                      const int32_t* __restrict__ aux, const double* __restrict__ V0,
                      double* __restrict__ b)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (i >= nunk) return;
    double v = 0.0;
    if (i < np && kind[i] == BEM_CONDUCTOR) v = V0[(int64_t)r * nregions + aux[i]];
    b[(int64_t)r * nunk + i] = v;
}

// Field at arbitrary points: one warp per point.  The warp scans all triangles
// with the classification of the regular pass (so that every pair is taken
// exactly once), gathers the near ones in shared memory and evaluates them 32 at
// a time with the FP64 closed form; then adds the far partials of all splits.
// perm (or NULL): point t's results go to slot perm[t] of phi and E.  In the FP32
// classification the warp first tests 32 chunk spheres at a time (a chunk of 32
// triangles whose sphere -- circumcentres plus eta R, with the rounding margin of
// k_far32p's unmasked chunks -- lies certainly outside the point holds no near
// triangle) and scans only the triangles of the other chunks, in the same ascending
// order, so the near list is unchanged.
template <bool F32>
__global__ void k_points_near(int64_t M, int64_t np, int splits, const double* __restrict__ pts,
                              const float4* __restrict__ chunk_sph,
                              const float4* __restrict__ hdr32, const double4* __restrict__ hdr64,
                              const double* __restrict__ geo, const double* __restrict__ u,
                              const double* __restrict__ part, double* __restrict__ phi,
                              double* __restrict__ E, unsigned long long* __restrict__ near_count,
                              const int32_t* __restrict__ perm)
{
    constexpr int WARPS = 4;
    __shared__ int32_t s_list[WARPS][64];
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int64_t t = blockIdx.x * (int64_t)WARPS + w;
    if (t >= M) return;
    const double x = pts[3 * t], y = pts[3 * t + 1], z = pts[3 * t + 2];
    const float xf = __double2float_rn(x), yf = __double2float_rn(y), zf = __double2float_rn(z);
    double p = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
    int n = 0, total = 0;
    auto flush = [&](int cnt) {
        if (lane < cnt) {
            const int32_t j = s_list[w][lane];
            double S, Gx, Gy, Gz;
            tri_closed_form(geo + GEO_STRIDE * (int64_t)j, x, y, z, false, S, Gx, Gy, Gz);
            const double uj = u[j];
            p = fma(uj, S, p);
            ex = fma(uj, Gx, ex);
            ey = fma(uj, Gy, ey);
            ez = fma(uj, Gz, ez);
        }
    };
    // scan the 32 triangles from j0: list the near ones, evaluate every full 32
    auto scan = [&](int64_t j0) {
        const int64_t j = j0 + lane;
        bool near = false;
        if (j < np) near = F32 ? !is_far32(xf, yf, zf, hdr32[j]) : !is_far64(x, y, z, hdr64[j]);
        const unsigned m = __ballot_sync(0xffffffffu, near);
        if (near) s_list[w][n + __popc(m & ((1u << lane) - 1u))] = (int32_t)j;
        n += __popc(m);
        total += __popc(m);
        __syncwarp();
        if (n >= 32) {
            flush(32);
            __syncwarp();
            if (lane < n - 32) s_list[w][lane] = s_list[w][lane + 32];
            __syncwarp();
            n -= 32;
        }
    };
    if (F32 && chunk_sph) {
        const int64_t nch = (np + 31) / 32;
        for (int64_t c0 = 0; c0 < nch; c0 += 32) {
            bool maybe = false;
            if (c0 + lane < nch) {
                const float4 cs = chunk_sph[c0 + lane];
                const float dx = xf - cs.x, dy = yf - cs.y, dz = zf - cs.z;
                maybe = !(sqrtf(dx * dx + dy * dy + dz * dz) > cs.w);
            }
            unsigned mm = __ballot_sync(0xffffffffu, maybe);
            while (mm) {
                const int b = __ffs(mm) - 1;
                mm &= mm - 1u;
                scan((c0 + b) * 32);
            }
        }
    } else {
        for (int64_t j0 = 0; j0 < np; j0 += 32) scan(j0);
    }
    flush(n);
    double fp = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
    for (int s = lane; s < splits; s += 32) {
        const double* q = part + ((int64_t)s * M + t) * 4;
        fp += q[0]; fx += q[1]; fy += q[2]; fz += q[3];
    }
    p = warp_sum(p) + kInv4Pi * warp_sum(fp);
    ex = warp_sum(ex) + kInv4Pi * warp_sum(fx);
    ey = warp_sum(ey) + kInv4Pi * warp_sum(fy);
    ez = warp_sum(ez) + kInv4Pi * warp_sum(fz);
    if (lane == 0) {
        atomicAdd(near_count, (unsigned long long)total);
        const int64_t o = perm ? (int64_t)perm[t] : t;
        if (phi) phi[o] = p;
        if (E) { E[3 * o] = ex; E[3 * o + 1] = ey; E[3 * o + 2] = ez; }
    }
}

// Dense rows, regular entries: one thread per (row, column).  Near entries are
// left for k_assemble_near.
template <bool F32, int Q>
__global__ void k_assemble_far(int64_t row0, int64_t nrows, int64_t np, int64_t lda,
                               const float4* __restrict__ tgt32, const double4* __restrict__ tgt64,
                               const float4* __restrict__ hdr32, const double4* __restrict__ hdr64,
                               const float4* __restrict__ node32, const double4* __restrict__ node64,
                               const double* __restrict__ geo, const int32_t* __restrict__ kind,
                               const double* __restrict__ rb, double* __restrict__ A)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t r = blockIdx.y;
    const int64_t i = row0 + r;
    if (j >= lda || r >= nrows) return;
    double* out = A + r * lda + j;
    if (j >= np || i >= np) { *out = 0.0; return; }
    double S = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
    bool far;
    if (F32) {
        const float4 t = tgt32[i];
        far = is_far32(t.x, t.y, t.z, hdr32[j]);
        if (far) {
            float s = 0.f, ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const float4 nd = node32[j * Q + k];
                const float dx = t.x - nd.x, dy = t.y - nd.y, dz = t.z - nd.z;
                const float ri = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                const float w = nd.w * ri, w3 = w * ri * ri;
                s += w; ax += w3 * dx; ay += w3 * dy; az += w3 * dz;
            }
            S = s; gx = ax; gy = ay; gz = az;
        }
    } else {
        const double4 t = tgt64[i];
        far = is_far64(t.x, t.y, t.z, hdr64[j]);
        if (far) {
#pragma unroll
            for (int k = 0; k < Q; ++k) {
                const double4 nd = node64[j * Q + k];
                const double dx = t.x - nd.x, dy = t.y - nd.y, dz = t.z - nd.z;
                const double ri = rsqrt(fma(dx, dx, fma(dy, dy, dz * dz)));
                const double w = nd.w * ri, w3 = w * ri * ri;
                S += w; gx += w3 * dx; gy += w3 * dy; gz += w3 * dz;
            }
        }
    }
    if (!far) return;
    S *= kInv4Pi; gx *= kInv4Pi; gy *= kInv4Pi; gz *= kInv4Pi;
    const double* gi = geo + GEO_STRIDE * i;
    const double en = gx * gi[GEO_N] + gy * gi[GEO_N + 1] + gz * gi[GEO_N + 2];
    *out = kind[i] == BEM_DIELECTRIC ? rb[i] * en : S;
}

// Dense rows, near entries, the diagonal term of dielectric rows and the -1 of
// the floating potential.  One warp per row.
__global__ void k_assemble_near(int64_t row0, int64_t nrows, int64_t np, int64_t lda,
                                const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                const double4* __restrict__ val, const uint8_t* __restrict__ flag,
                                uint8_t bit, const double* __restrict__ geo,
                                const int32_t* __restrict__ kind, const int32_t* __restrict__ aux,
                                const double* __restrict__ ra, const double* __restrict__ rb,
                                double* __restrict__ A)
{
    const int lane = threadIdx.x & 31;
    const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (r >= nrows) return;
    const int64_t i = row0 + r;
    if (i >= np) return;
    const double* gi = geo + GEO_STRIDE * i;
    const int kd = kind[i];
    for (int64_t k = ptr[i] + lane; k < ptr[i + 1]; k += 32) {
        if (!(flag[k] & bit)) continue;
        const int32_t j = col[k];
        const double4 v = val[k];
        const double en = v.y * gi[GEO_N] + v.z * gi[GEO_N + 1] + v.w * gi[GEO_N + 2];
        double a = kd == BEM_DIELECTRIC ? rb[i] * en : v.x;
        if (kd == BEM_DIELECTRIC && j == i) a += ra[i];
        A[r * lda + j] = a;
    }
    if (lane == 0 && kd == BEM_FLOATING) A[r * lda + np + aux[i]] = -1.0;
}

// Neutrality rows (Eq. Final4): one thread per column j, summing over the rows
// of the floating body; regular pairs by the rule, near pairs looked up in the
// row's sorted near list.
template <bool F32, int Q>
__global__ void k_assemble_neutral(int f, int64_t np, const int32_t* __restrict__ rows,
                                   const int32_t* __restrict__ off, const float4* __restrict__ tgt32,
                                   const double4* __restrict__ tgt64, const float4* __restrict__ hdr32,
                                   const double4* __restrict__ hdr64, const float4* __restrict__ node32,
                                   const double4* __restrict__ node64, const double* __restrict__ geo,
                                   const int64_t* __restrict__ ptr, const int32_t* __restrict__ col,
                                   const double4* __restrict__ val, const uint8_t* __restrict__ flag,
                                   uint8_t bit, const double* __restrict__ rw,
                                   const double* __restrict__ rs, double* __restrict__ out)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= np) return;
    double acc = 0.0;
    for (int k = off[f]; k < off[f + 1]; ++k) {
        const int64_t i = rows[k];
        const double* gi = geo + GEO_STRIDE * i;
        double gx = 0.0, gy = 0.0, gz = 0.0;
        bool near;
        if (F32) {
            const float4 t = tgt32[i];
            near = !is_far32(t.x, t.y, t.z, hdr32[j]);
            if (!near) {
                float ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const float4 nd = node32[j * Q + q];
                    const float dx = t.x - nd.x, dy = t.y - nd.y, dz = t.z - nd.z;
                    const float ri = rsqrtf(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
                    const float w3 = nd.w * ri * ri * ri;
                    ax += w3 * dx; ay += w3 * dy; az += w3 * dz;
                }
                gx = ax * kInv4Pi; gy = ay * kInv4Pi; gz = az * kInv4Pi;
            }
        } else {
            const double4 t = tgt64[i];
            near = !is_far64(t.x, t.y, t.z, hdr64[j]);
            if (!near) {
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const double4 nd = node64[j * Q + q];
                    const double dx = t.x - nd.x, dy = t.y - nd.y, dz = t.z - nd.z;
                    const double ri = rsqrt(fma(dx, dx, fma(dy, dy, dz * dz)));
                    const double w3 = nd.w * ri * ri * ri;
                    gx += w3 * dx; gy += w3 * dy; gz += w3 * dz;
                }
                gx *= kInv4Pi; gy *= kInv4Pi; gz *= kInv4Pi;
            }
        }
        if (near) {
            int64_t lo = ptr[i], hi = ptr[i + 1];
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (col[mid] < j) lo = mid + 1; else hi = mid;
            }
            if (lo < ptr[i + 1] && col[lo] == j && (flag[lo] & bit)) {
                const double4 v = val[lo];
                gx = v.y; gy = v.z; gz = v.w;
            }
        }
        double en = gx * gi[GEO_N] + gy * gi[GEO_N + 1] + gz * gi[GEO_N + 2];
        if (j == i) en += 0.5;
        acc += rw[i] * en;
        if (j == i) acc += rs[i];  // a sheet's eps- u_i term (Eq. sheets)
    }
    out[j] = acc;
}

template <bool F32>
int assemble_dispatch(bem_ctx* c, int64_t row0, int64_t row1, double* A, int64_t lda)
{
    const int64_t nrows = row1 - row0;
    const int64_t np = c->np;
    const uint8_t bit = F32 ? 1 : 2;
    cudaStream_t s = c->stream;
    if (nrows <= 0) return BEM_OK;
    // zero-fill + regular entries, in row batches of at most 65535 (grid.y)
    for (int64_t rb0 = 0; rb0 < nrows; rb0 += 65535) {
        const int64_t nb = std::min<int64_t>(65535, nrows - rb0);
        dim3 grid((unsigned)((lda + 127) / 128), (unsigned)nb);
#define ASM_FAR(QQ)                                                                              \
    k_assemble_far<F32, QQ><<<grid, 128, 0, s>>>(row0 + rb0, nb, np, lda, c->tgt32, c->tgt64,    \
                                                 c->hdr32, c->hdr64, c->node32, c->node64, c->geo, \
                                                 c->row_kind, c->row_b, A + rb0 * lda)
        switch (c->g) {
            case 1: ASM_FAR(1); break;
            case 2: ASM_FAR(4); break;
            case 3: ASM_FAR(9); break;
            case 4: ASM_FAR(16); break;
            case 5: ASM_FAR(25); break;
            case 6: ASM_FAR(36); break;
            default: return set_err(c, BEM_ERR_ARG, "far_order %d not compiled", c->g);
        }
#undef ASM_FAR
        BEM_LAUNCH_CHECK(c);
    }
    k_assemble_near<<<(unsigned)((nrows * 32 + 127) / 128), 128, 0, s>>>(
        row0, nrows, np, lda, c->near_ptr, c->near_col, c->near_val, c->near_flag, bit, c->geo,
        c->row_kind, c->row_aux, c->row_a, c->row_b, A);
    BEM_LAUNCH_CHECK(c);
    for (int f = 0; f < c->nfloat; ++f) {
        const int64_t r = np + f;
        if (r < row0 || r >= row1) continue;
        double* out = A + (r - row0) * lda;
        BEM_CUDA_TRY(c, cudaMemsetAsync(out, 0, lda * sizeof(double), s));
#define ASM_NEU(QQ)                                                                             \
    k_assemble_neutral<F32, QQ><<<(unsigned)((np + 127) / 128), 128, 0, s>>>(                    \
        f, np, c->float_rows, c->float_off, c->tgt32, c->tgt64, c->hdr32, c->hdr64, c->node32,  \
        c->node64, c->geo, c->near_ptr, c->near_col, c->near_val, c->near_flag, bit, c->row_w, c->row_s, out)
        switch (c->g) {
            case 1: ASM_NEU(1); break;
            case 2: ASM_NEU(4); break;
            case 3: ASM_NEU(9); break;
            case 4: ASM_NEU(16); break;
            case 5: ASM_NEU(25); break;
            case 6: ASM_NEU(36); break;
            default: return set_err(c, BEM_ERR_ARG, "far_order %d not compiled", c->g);
        }
#undef ASM_NEU
        BEM_LAUNCH_CHECK(c);
    }
    return BEM_OK;
}

}  // namespace

int matvec_impl(bem_ctx* c, int precision, int nrhs, const double* x, double* y, bool need_E)
{
    if (c->p1) return p1_matvec_impl(c, precision, nrhs, x, y);
    const int64_t np = c->np, n = c->nunk;
    const int splits = far_splits(c, precision, np);
    if ((size_t)splits * np * 4 * nrhs > c->part_cap)
        return set_err(c, BEM_ERR_CAPACITY, "far workspace too small");
    FarTargets T{c->tgt32, c->tgt_lo32, c->tgt64, nullptr, np, need_E ? nullptr : c->row_kind};
    int rc = launch_far(c, precision, T, x, nrhs, n, splits, c->part);
    if (rc) return rc;
    c->cnt.matvecs[precision] += nrhs;
    // near pairs: the FP32 / FP64 classification's closed forms; the double-FP32
    // pass masks like FP32 and takes the corrected values that reproduce FP64
    const uint8_t bit = precision == BEM_MIXED ? 1 : (precision == BEM_FP64 ? 2 : 3);
    const double4* nval = precision == kPrecDF ? c->near_val_df : c->near_val;
    for (int r = 0; r < nrhs; ++r) {
        const double* pr = c->part + (size_t)r * splits * np * 4;
        k_rows<<<(unsigned)((np * 32 + 127) / 128), 128, 0, c->stream>>>(
            np, splits, pr, c->near_ptr, c->near_col, nval, c->near_flag, bit, x + r * n,
            c->geo, c->row_kind, c->row_aux, c->row_a, c->row_b, c->row_w, c->row_s, 0, y + r * n,
            c->neut + r * np, c->field + (size_t)r * np * 4);
        BEM_LAUNCH_CHECK(c);
        if (c->nfloat > 0) {
            k_neutrality<<<c->nfloat, kNeutThreads, 0, c->stream>>>(np, c->float_rows, c->float_off,
                                                            c->neut + r * np, y + r * n);
            BEM_LAUNCH_CHECK(c);
        }
    }
    return BEM_OK;
}

static int check_prec(bem_ctx* c, int precision)
{
    if (precision != BEM_FP64 && precision != BEM_MIXED)
        return set_err(c, BEM_ERR_ARG, "precision must be BEM_FP64 or BEM_MIXED");
    return BEM_OK;
}

extern "C" int bem_matvec(bem_ctx* c, int32_t precision, int32_t nrhs, const double* x, double* y)
{
    if (!c) return BEM_ERR_ARG;
    if (precision != BEM_DF)
        if (int rc = check_prec(c, precision)) return rc;
    if (nrhs < 1 || nrhs > kMaxRhs || !x || !y)
        return set_err(c, BEM_ERR_ARG, "bem_matvec: need 1 <= nrhs <= %d and non-NULL x, y", kMaxRhs);
    if (c->p1 && precision == BEM_DF)
        return set_err(c, BEM_ERR_ARG, "bem_matvec: BEM_DF is not built for curved triangles");
    return matvec_impl(c, precision, nrhs, x, y);
}

extern "C" int bem_rhs(bem_ctx* c, int32_t nrhs, const double* V0, double* b)
{
    if (!c) return BEM_ERR_ARG;
    if (nrhs < 1 || nrhs > kMaxRhs || !b) return set_err(c, BEM_ERR_ARG, "bem_rhs: bad nrhs or b");
    const int nreg = (int)c->regions.size();
    const double* v = V0 ? V0 : c->region_V0;
    if (!V0 && nrhs != 1) return set_err(c, BEM_ERR_ARG, "bem_rhs: V0 = NULL needs nrhs = 1");
    if (c->p1) return p1_rhs(c, nrhs, V0, b);
    dim3 grid((unsigned)((c->nunk + 255) / 256), (unsigned)nrhs);
    k_rhs<<<grid, 256, 0, c->stream>>>(c->np, c->nunk, nreg, c->row_kind, c->row_aux, v, b);
    BEM_LAUNCH_CHECK(c);
    return BEM_OK;
}

extern "C" int bem_surface_field(bem_ctx* c, int32_t precision, const double* u, double* E)
{
    if (!c) return BEM_ERR_ARG;
    if (int rc = check_prec(c, precision)) return rc;
    if (!u || !E) return set_err(c, BEM_ERR_ARG, "bem_surface_field: NULL pointer");
    if (c->p1) return set_err(c, BEM_ERR_ARG, "bem_surface_field: not built for curved triangles");
    const int64_t np = c->np;
    const int splits = far_splits(c, precision, np);
    FarTargets T{c->tgt32, c->tgt_lo32, c->tgt64, nullptr, np};
    int rc = launch_far(c, precision, T, u, 1, 0, splits, c->part);
    if (rc) return rc;
    const uint8_t bit = precision == BEM_MIXED ? 1 : 2;
    k_rows<<<(unsigned)((np * 32 + 127) / 128), 128, 0, c->stream>>>(
        np, splits, c->part, c->near_ptr, c->near_col, c->near_val, c->near_flag, bit, u, c->geo,
        c->row_kind, c->row_aux, c->row_a, c->row_b, c->row_w, c->row_s, 1, E, nullptr, nullptr);
    BEM_LAUNCH_CHECK(c);
    return BEM_OK;
}

// Deferred near pass + split reduction for M points whose far partial sums are in
// part[splits][M][4] (used by the static-scratch entry point).
int launch_points_near(bem_ctx* c, int precision, int64_t M, const double* pts, const double* u,
                       const double* part, int splits, double* phi, double* E)
{
    if (M <= 0) return BEM_OK;
    const unsigned blocks = (unsigned)((M + 3) / 4);
    if (precision == BEM_MIXED)
        k_points_near<true><<<blocks, 128, 0, c->stream>>>(M, c->np, splits, pts, c->chunk_sph, c->hdr32,
                                                             c->hdr64, c->geo, u, part, phi, E,
                                                             c->d_near_count + BEM_MIXED, nullptr);
    else
        k_points_near<false><<<blocks, 128, 0, c->stream>>>(M, c->np, splits, pts, nullptr, c->hdr32,
                                                              c->hdr64, c->geo, u, part, phi, E,
                                                              c->d_near_count + BEM_FP64, nullptr);
    BEM_LAUNCH_CHECK(c);
    return BEM_OK;
}

extern "C" int bem_eval_field(bem_ctx* c, int32_t precision, const double* u, int64_t M,
                              const double* pts, double* phi, double* E)
{
    if (!c) return BEM_ERR_ARG;
    if (int rc = check_prec(c, precision)) return rc;
    if (M < 0 || (M > 0 && (!u || !pts))) return set_err(c, BEM_ERR_ARG, "bem_eval_field: bad M or NULL");
    if (c->p1) return M > 0 ? p1_eval_field(c, precision, u, M, pts, phi, E) : BEM_OK;
    const int64_t CH = c->prm.max_points;
    for (int64_t m0 = 0; m0 < M; m0 += CH) {
        const int64_t mc = std::min(CH, M - m0);
        const int splits = far_splits(c, precision, mc);
        if ((size_t)splits * mc * 4 > c->part_cap)
            return set_err(c, BEM_ERR_CAPACITY, "far workspace too small");
        // the packed FP32 kernel takes the chunk's points in spatial order (order.cu):
        // its tiles of consecutive points are then compact, so most triangle chunks
        // are summed without per-pair classification
        const double* cp = pts + 3 * m0;
        const int32_t* perm = nullptr;
        if (precision == BEM_MIXED && c->far32_tp >= 2 && mc >= kOrderMin) {
            if (int rc = order_points(c, mc, cp, c->ord_pts, c->ord_perm)) return rc;
            cp = c->ord_pts;
            perm = c->ord_perm;
        }
        FarTargets T{nullptr, nullptr, nullptr, cp, mc};
        int rc = launch_far(c, precision, T, u, 1, 0, splits, c->part);
        if (rc) return rc;
        const unsigned blocks = (unsigned)((mc + 3) / 4);
        if (precision == BEM_MIXED)
            k_points_near<true><<<blocks, 128, 0, c->stream>>>(
                mc, c->np, splits, cp, c->chunk_sph, c->hdr32, c->hdr64, c->geo, u, c->part,
                phi ? phi + m0 : nullptr, E ? E + 3 * m0 : nullptr, c->d_near_count + BEM_MIXED, perm);
        else
            k_points_near<false><<<blocks, 128, 0, c->stream>>>(
                mc, c->np, splits, cp, nullptr, c->hdr32, c->hdr64, c->geo, u, c->part,
                phi ? phi + m0 : nullptr, E ? E + 3 * m0 : nullptr, c->d_near_count + BEM_FP64, perm);
        BEM_LAUNCH_CHECK(c);
    }
    return BEM_OK;
}

extern "C" int bem_assemble_rows(bem_ctx* c, int64_t row0, int64_t row1, int32_t precision,
                                 double* A, int64_t lda)
{
    if (!c) return BEM_ERR_ARG;
    if (int rc = check_prec(c, precision)) return rc;
    if (row0 < 0 || row1 < row0 || row1 > c->nunk || lda < c->nunk || (!A && row1 > row0))
        return set_err(c, BEM_ERR_ARG, "bem_assemble_rows: bad rows [%lld,%lld) or lda",
                       (long long)row0, (long long)row1);
    if (c->p1) return p1_assemble(c, row0, row1, precision, A, lda);
    return precision == BEM_MIXED ? assemble_dispatch<true>(c, row0, row1, A, lda)
                                  : assemble_dispatch<false>(c, row0, row1, A, lda);
}

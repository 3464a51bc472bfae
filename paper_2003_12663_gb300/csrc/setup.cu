// setup.cu -- context creation: quadrature rule, per-triangle precompute (Sec. 4:
// "circumcenters and circumradii of the triangles can be precomputed"), the near
// pairs of the collocation points with their closed-form values, row data of
// Eqs. Final1-Final4 and the fixed workspace.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>

#include "bem_internal.cuh"

static std::string g_create_err;

int set_err(bem_ctx* ctx, int code, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx)
        ctx->err = buf;
    else
        g_create_err = buf;
    return code;
}

// ---------------------------------------------------------------- Gauss rules
// n-point Gauss-Legendre on [-1,1]: Newton's method on P_n, evaluated by the
// three-term recurrence (k+1) P_{k+1} = (2k+1) z P_k - k P_{k-1}.
void gauss_legendre_pm1(int n, std::vector<double>& x, std::vector<double>& w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) {
                // one more evaluation at the converged root for the weight
                p0 = 1.0; p1 = z;
                for (int k = 2; k <= n; ++k) {
                    const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                    p0 = p1;
                    p1 = p2;
                }
                dp = n * (z * p1 - p0) / (z * z - 1.0);
                break;
            }
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// n-point Gauss rule on [0,1] for the weight u^weight_power (0 or 1):
// recurrence coefficients of the monic orthogonal polynomials by the Stieltjes
// procedure on a 64-point Gauss-Legendre rule (exact for these weights up to
// n = 8), roots by bisection on sign changes, weights by the Christoffel numbers
// lambda_i = 1 / sum_k p_k(x_i)^2 / ||p_k||^2.
void host_gauss_rule(int n, int weight_power, std::vector<double>& xo, std::vector<double>& wo)
{
    std::vector<double> bx, bw;
    gauss_legendre_pm1(64, bx, bw);
    const int B = (int)bx.size();
    std::vector<double> t(B), W(B);
    for (int i = 0; i < B; ++i) {
        t[i] = 0.5 * (bx[i] + 1.0);
        W[i] = 0.5 * bw[i] * (weight_power ? t[i] : 1.0);
    }
    std::vector<double> a(n), b(n), nrm(n);
    std::vector<double> pprev(B, 0.0), pcur(B, 1.0), pnext(B);
    double nprev = 1.0;
    for (int k = 0; k < n; ++k) {
        double s0 = 0.0, s1 = 0.0;
        for (int i = 0; i < B; ++i) {
            s0 += W[i] * pcur[i] * pcur[i];
            s1 += W[i] * t[i] * pcur[i] * pcur[i];
        }
        nrm[k] = s0;
        a[k] = s1 / s0;
        b[k] = (k == 0) ? 0.0 : s0 / nprev;
        for (int i = 0; i < B; ++i) pnext[i] = (t[i] - a[k]) * pcur[i] - b[k] * pprev[i];
        pprev.swap(pcur);
        pcur.swap(pnext);
        nprev = s0;
    }
    auto pn = [&](double z, std::vector<double>* vals) {
        double p0 = 0.0, p1 = 1.0;
        if (vals) (*vals)[0] = 1.0;
        for (int k = 0; k < n; ++k) {
            const double p2 = (z - a[k]) * p1 - b[k] * p0;
            p0 = p1;
            p1 = p2;
            if (vals && k + 1 < n) (*vals)[k + 1] = p1;
        }
        return p1;
    };
    xo.clear();
    wo.clear();
    const int G = 4096;
    double zl = 0.0, fl = pn(0.0, nullptr);
    for (int s = 1; s <= G && (int)xo.size() < n; ++s) {
        const double zr = (double)s / G, fr = pn(zr, nullptr);
        if ((fl < 0.0) != (fr < 0.0)) {
            double lo = zl, hi = zr, flo = fl;
            for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
                const double mid = 0.5 * (lo + hi);
                if (mid <= lo || mid >= hi) break;
                const double fm = pn(mid, nullptr);
                if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; } else { hi = mid; }
            }
            xo.push_back(0.5 * (lo + hi));
        }
        zl = zr;
        fl = fr;
    }
    std::vector<double> vals(n);
    for (double z : xo) {
        pn(z, &vals);
        double s = 0.0;
        for (int k = 0; k < n; ++k) s += vals[k] * vals[k] / nrm[k];
        wo.push_back(1.0 / s);
    }
}

// ---------------------------------------------------------------- kernels
__constant__ double c_rule_u[kMaxOrder], c_rule_wu[kMaxOrder], c_rule_v[kMaxOrder],
    c_rule_wv[kMaxOrder];

// One thread per triangle: geometry record, classification header and the
// Duffy/Gauss nodes y(u,v) = a + u (b - a) + u v (c - b), weight 2A lambda_k w_l
// (lambda: rule for the weight u, which carries the Duffy Jacobian).
__global__ void k_panels(int64_t np, int g, double eta, const double* __restrict__ X,
                         const int32_t* __restrict__ tri, double* __restrict__ geo,
                         float4* __restrict__ hdr32, double4* __restrict__ hdr64,
                         float4* __restrict__ node32, double4* __restrict__ node64,
                         float4* __restrict__ tgt32, double4* __restrict__ tgt64,
                         float4* __restrict__ node_lo32, float4* __restrict__ tgt_lo32,
                         int* __restrict__ status)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= np) return;
    double v[9];
    for (int k = 0; k < 3; ++k) {
        const int64_t vi = tri[3 * j + k];
        v[3 * k] = X[3 * vi];
        v[3 * k + 1] = X[3 * vi + 1];
        v[3 * k + 2] = X[3 * vi + 2];
    }
    const double abx = v[3] - v[0], aby = v[4] - v[1], abz = v[5] - v[2];
    const double bcx = v[6] - v[3], bcy = v[7] - v[4], bcz = v[8] - v[5];
    const double cax = v[0] - v[6], cay = v[1] - v[7], caz = v[2] - v[8];
    // n ~ (b-a) x (c-a) = (b-a) x (b-a + c-b) = (b-a) x (c-b)
    const double wx = aby * bcz - abz * bcy, wy = abz * bcx - abx * bcz, wz = abx * bcy - aby * bcx;
    const double wn = sqrt(wx * wx + wy * wy + wz * wz);
    double* gp = geo + GEO_STRIDE * j;
    if (!(wn > 0.0)) {
        atomicExch(status, BEM_ERR_DEGENERATE);
        for (int k = 0; k < GEO_STRIDE; ++k) gp[k] = 0.0;
        return;
    }
    for (int k = 0; k < 9; ++k) gp[k] = v[k];
    gp[GEO_N] = wx / wn;
    gp[GEO_N + 1] = wy / wn;
    gp[GEO_N + 2] = wz / wn;
    const double area = 0.5 * wn;
    gp[GEO_AREA] = area;
    const double cx = (v[0] + v[3] + v[6]) / 3.0, cy = (v[1] + v[4] + v[7]) / 3.0,
                 cz = (v[2] + v[5] + v[8]) / 3.0;
    gp[GEO_CTR] = cx;
    gp[GEO_CTR + 1] = cy;
    gp[GEO_CTR + 2] = cz;
    // circumcentre from barycentric weights la (lb+lc-la) etc., la = |b-c|^2 opposite a
    const double la = bcx * bcx + bcy * bcy + bcz * bcz;
    const double lb = cax * cax + cay * cay + caz * caz;
    const double lc = abx * abx + aby * aby + abz * abz;
    const double wa = la * (lb + lc - la), wb = lb * (lc + la - lb), wc = lc * (la + lb - lc);
    const double ws = wa + wb + wc;
    const double ccx = (wa * v[0] + wb * v[3] + wc * v[6]) / ws;
    const double ccy = (wa * v[1] + wb * v[4] + wc * v[7]) / ws;
    const double ccz = (wa * v[2] + wb * v[5] + wc * v[8]) / ws;
    const double R = sqrt(la * lb * lc) / (4.0 * area);
    gp[GEO_CC] = ccx;
    gp[GEO_CC + 1] = ccy;
    gp[GEO_CC + 2] = ccz;
    gp[GEO_R] = R;
    gp[GEO_ETAR] = eta * R;
    gp[21] = gp[22] = gp[23] = 0.0;
    const double eR2 = (eta * R) * (eta * R);
    hdr64[j] = make_double4(ccx, ccy, ccz, eR2);
    hdr32[j] = make_float4(__double2float_rn(ccx), __double2float_rn(ccy), __double2float_rn(ccz),
                           __double2float_rn(eR2));
    tgt64[j] = make_double4(cx, cy, cz, 0.0);
    tgt32[j] = make_float4(__double2float_rn(cx), __double2float_rn(cy), __double2float_rn(cz), 0.f);
    {
        const float4 h = tgt32[j];
        tgt_lo32[j] = make_float4(__double2float_rn(cx - (double)h.x), __double2float_rn(cy - (double)h.y),
                                  __double2float_rn(cz - (double)h.z), 0.f);
    }
    const int Q = g * g;
    for (int k = 0; k < g; ++k) {
        const double uk = c_rule_u[k];
        for (int l = 0; l < g; ++l) {
            const double vl = c_rule_v[l];
            const double yx = v[0] + uk * abx + uk * vl * bcx;
            const double yy = v[1] + uk * aby + uk * vl * bcy;
            const double yz = v[2] + uk * abz + uk * vl * bcz;
            const double w = 2.0 * area * c_rule_wu[k] * c_rule_wv[l];
            node64[j * Q + k * g + l] = make_double4(yx, yy, yz, w);
            const float4 h = make_float4(__double2float_rn(yx), __double2float_rn(yy),
                                         __double2float_rn(yz), __double2float_rn(w));
            node32[j * Q + k * g + l] = h;
            node_lo32[j * Q + k * g + l] =
                make_float4(__double2float_rn(yx - (double)h.x), __double2float_rn(yy - (double)h.y),
                            __double2float_rn(yz - (double)h.z), __double2float_rn(w - (double)h.w));
        }
    }
}

// Per triangle for the field-line integrator: the unit normal rounded to FP32 and
// the region index (as the bits of w), so that one 16-byte record carries what the
// electrode indicator needs.
__global__ void k_nrm32(int64_t np, const double* __restrict__ geo, const int32_t* __restrict__ region,
                        float4* __restrict__ out)
{
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= np) return;
    const double* g = geo + GEO_STRIDE * j;
    out[j] = make_float4(__double2float_rn(g[GEO_N]), __double2float_rn(g[GEO_N + 1]),
                         __double2float_rn(g[GEO_N + 2]), __int_as_float(region[j]));
}

// Bounding sphere of the near zones |x - cc_j| <= eta R_j of 32 consecutive
// triangles, enlarged by a margin that covers the FP32 rounding of the
// classification: a target farther than the radius from the centre is regular
// for all 32 triangles in every kernel of the FP32 form.
__global__ void k_chunk_spheres(int64_t np, const double* __restrict__ geo, float4* __restrict__ sph)
{
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t j0 = c * 32, j1 = min(np, j0 + 32);
    if (j0 >= np) return;
    double cx = 0.0, cy = 0.0, cz = 0.0;
    for (int64_t j = j0; j < j1; ++j) {
        const double* g = geo + GEO_STRIDE * j;
        cx += g[GEO_CC]; cy += g[GEO_CC + 1]; cz += g[GEO_CC + 2];
    }
    const double inv = 1.0 / (double)(j1 - j0);
    cx *= inv; cy *= inv; cz *= inv;
    double r = 0.0;
    for (int64_t j = j0; j < j1; ++j) {
        const double* g = geo + GEO_STRIDE * j;
        const double dx = g[GEO_CC] - cx, dy = g[GEO_CC + 1] - cy, dz = g[GEO_CC + 2] - cz;
        r = fmax(r, sqrt(dx * dx + dy * dy + dz * dz) + g[GEO_ETAR]);
    }
    const double mag = fmax(fabs(cx), fmax(fabs(cy), fabs(cz)));
    r += 1e-5 * (r + mag) + 1e-30;
    sph[c] = make_float4(__double2float_rn(cx), __double2float_rn(cy), __double2float_rn(cz),
                         __double2float_ru(r));
}

// One warp per collocation row: count (phase 0) or list (phase 1) the triangles
// that are near in the FP32 or the FP64 classification.  Columns ascend.
__global__ void k_near_rows(int64_t np, int phase, const float4* __restrict__ tgt32,
                            const double4* __restrict__ tgt64, const float4* __restrict__ hdr32,
                            const double4* __restrict__ hdr64, int32_t* __restrict__ count,
                            const int64_t* __restrict__ ptr, int32_t* __restrict__ col,
                            uint8_t* __restrict__ flag)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= np) return;
    const float4 t32 = tgt32[i];
    const double4 t64 = tgt64[i];
    int64_t pos = phase ? ptr[i] : 0;
    int cnt = 0;
    for (int64_t j0 = 0; j0 < np; j0 += 32) {
        const int64_t j = j0 + lane;
        bool n32 = false, n64 = false;
        if (j < np) {
            n32 = !is_far32(t32.x, t32.y, t32.z, hdr32[j]);
            n64 = !is_far64(t64.x, t64.y, t64.z, hdr64[j]);
        }
        const unsigned m = __ballot_sync(0xffffffffu, n32 || n64);
        if (phase && (n32 || n64)) {
            const int r = __popc(m & ((1u << lane) - 1u));
            col[pos + r] = (int32_t)j;
            flag[pos + r] = (uint8_t)((n32 ? 1 : 0) | (n64 ? 2 : 0));
        }
        pos += __popc(m);
        cnt += __popc(m);
    }
    if (!phase && lane == 0) count[i] = cnt;
}

// One thread per near pair: exact S and G (principal value of the own panel).
//
// The double-FP32 residual pass masks near pairs with the FP32 classification but
// must reproduce the FP64 form, so its near values are
//   val_df = [near in FP64] exact + ([far in FP64] - [far in FP32]) quad64,
// quad64 being the FP64 Duffy/Gauss value of the pair: "exact" where both agree,
// "exact - quad" where only FP64 calls the pair near (the pass added quad), "quad"
// where only FP32 does (the pass skipped a pair the FP64 form integrates).
__global__ void k_near_values(int64_t np, int Q, const int64_t* __restrict__ ptr,
                              const int32_t* __restrict__ col, const uint8_t* __restrict__ flag,
                              const double* __restrict__ geo, const double4* __restrict__ node64,
                              double4* __restrict__ val, double4* __restrict__ val_df)
{
    const int64_t i = blockIdx.x;
    const double* gi = geo + GEO_STRIDE * i;
    const double x = gi[GEO_CTR], y = gi[GEO_CTR + 1], z = gi[GEO_CTR + 2];
    for (int64_t k = ptr[i] + threadIdx.x; k < ptr[i + 1]; k += blockDim.x) {
        const int32_t j = col[k];
        double S, Gx, Gy, Gz;
        tri_closed_form(geo + GEO_STRIDE * (int64_t)j, x, y, z, j == i, S, Gx, Gy, Gz);
        val[k] = make_double4(S, Gx, Gy, Gz);
        const bool n32 = flag[k] & 1, n64 = flag[k] & 2;
        double qS = 0.0, qx = 0.0, qy = 0.0, qz = 0.0;
        if (n32 != n64) {
            for (int q = 0; q < Q; ++q) {
                const double4 nd = node64[(int64_t)j * Q + q];
                const double dx = x - nd.x, dy = y - nd.y, dz = z - nd.z;
                const double ri = rsqrt(dx * dx + dy * dy + dz * dz);
                const double w = nd.w * ri, w3 = w * ri * ri;
                qS += w; qx += w3 * dx; qy += w3 * dy; qz += w3 * dz;
            }
            qS *= kInv4Pi; qx *= kInv4Pi; qy *= kInv4Pi; qz *= kInv4Pi;
        }
        const double a = n64 ? 1.0 : 0.0;
        const double b = (n64 ? 0.0 : 1.0) - (n32 ? 0.0 : 1.0);
        val_df[k] = make_double4(a * S + b * qS, a * Gx + b * qx, a * Gy + b * qy, a * Gz + b * qz);
    }
}

// Inverse Jacobi diagonal (Sec. 5: GMRES with a diagonal preconditioner).
// Conductor and floating rows: S_ii; dielectric rows: (eps+ + eps-)/2; the
// neutrality rows have no diagonal entry and take 1.
__global__ void k_jacobi(int64_t np, int64_t nunk, const int32_t* __restrict__ kind,
                         const double* __restrict__ row_a, const int64_t* __restrict__ ptr,
                         const int32_t* __restrict__ col, const double4* __restrict__ val,
                         double* __restrict__ jinv)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= nunk) return;
    double d = 1.0;
    if (i < np) {
        if (kind[i] == BEM_DIELECTRIC) {
            d = row_a[i];
        } else {
            for (int64_t k = ptr[i]; k < ptr[i + 1]; ++k)
                if (col[k] == i) d = val[k].x;
        }
    }
    jinv[i] = (d != 0.0) ? 1.0 / d : 1.0;
}

// ---------------------------------------------------------------- create / destroy
template <class T>
static int dalloc(bem_ctx* ctx, T** p, size_t n)
{
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return set_err(ctx, BEM_ERR_NOMEM, "cudaMalloc of %zu bytes failed: %s", n * sizeof(T),
                       cudaGetErrorString(e));
    }
    return BEM_OK;
}

static void free_ctx(bem_ctx* c)
{
    if (!c) return;
    adjoint_workspace_free(c);
    p1_free(c);
    void* ptrs[] = {c->X, c->tri, c->geo, c->hdr32, c->hdr64, c->node32, c->node64, c->tgt32,
                    c->tgt64, c->row_kind, c->row_aux, c->row_a, c->row_b, c->row_w, c->region_V0,
                    c->row_s, c->float_rows, c->float_off, c->jinv, c->near_ptr, c->near_col, c->near_val,
                    c->near_flag, c->part, c->field, c->neut, c->pts_stage, c->V, c->wvec,
                    c->zvec, c->rvec, c->bvec, c->dvec, c->ivec, c->hcol, c->d_status,
                    c->d_near_count, c->node_lo32, c->tgt_lo32, c->near_val_df, c->d_region,
                    c->d_electrode, c->qnode, c->chunk_sph, c->csc_ptr, c->csc_row, c->csc_ent,
                    c->tsrc64, c->tsrc32, c->nrm32, c->d_line_next, c->u32, c->ord_pts,
                    c->ord_perm, c->ord_cell, c->ord_hist, c->ord_box};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (c->hcol_host) cudaFreeHost(c->hcol_host);
    for (cudaEvent_t e : c->ev0)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : c->ev1)
        if (e) cudaEventDestroy(e);
    delete c;
}

// ---------------------------------------------------------------- counters, timing
// Events come from a fixed pool created at bem_create; when it is full, the
// pending intervals are summed (after a stream synchronisation) and reused.
static void timing_drain(bem_ctx* c)
{
    if (c->ev_used == 0) return;
    cudaStreamSynchronize(c->stream);
    for (size_t k = 0; k < c->ev_used; ++k) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev0[k], c->ev1[k]) == cudaSuccess)
            c->cnt.far_ms[c->ev_prec[k]] += ms;
        else
            cudaGetLastError();
    }
    c->ev_used = 0;
}

void timing_begin(bem_ctx* c, int precision)
{
    if (!c->prm.timing || c->ev0.empty()) return;
    if (c->ev_used == c->ev0.size()) timing_drain(c);
    c->ev_prec[c->ev_used] = precision;
    cudaEventRecord(c->ev0[c->ev_used], c->stream);
}

void timing_end(bem_ctx* c)
{
    if (!c->prm.timing || c->ev0.empty()) return;
    cudaEventRecord(c->ev1[c->ev_used], c->stream);
    ++c->ev_used;
}

extern "C" int bem_get_counters(bem_ctx* c, bem_counters* out)
{
    if (!c || !out) return BEM_ERR_ARG;
    timing_drain(c);
    BEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    unsigned long long nc[4] = {0, 0, 0, 0};
    BEM_CUDA_TRY(c, cudaMemcpy(nc, c->d_near_count, sizeof nc, cudaMemcpyDeviceToHost));
    *out = c->cnt;
    out->near_pairs[0] += (int64_t)nc[0];
    out->near_pairs[1] += (int64_t)nc[1];
    out->chunks32p = (int64_t)nc[2];
    out->fast_chunks32p = (int64_t)nc[3];
    return BEM_OK;
}

extern "C" int bem_reset_counters(bem_ctx* c)
{
    if (!c) return BEM_ERR_ARG;
    timing_drain(c);
    c->cnt = bem_counters{};
    c->cnt.far32_variant = c->far32_tp;
    BEM_CUDA_TRY(c, cudaMemsetAsync(c->d_near_count, 0, 4 * sizeof(unsigned long long), c->stream));
    BEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return BEM_OK;
}

extern "C" void bem_default_params(bem_params* p)
{
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->eta = 4.0;
    p->far_order = 3;
    p->gmres_restart = 100;
    p->max_iters = 2000;
    p->max_refine = 6;
    p->max_points = 131072;
    p->timing = 0;
    p->residual = BEM_RESIDUAL_DF_UPDATE;
    p->adjoint_checkpoint = 128;
    p->adjoint_lines = 256;
    p->trace_cluster = 0;
}

extern "C" const char* bem_last_error(const bem_ctx* ctx)
{
    return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

extern "C" int bem_sizes(const bem_ctx* ctx, int64_t* n_panels, int64_t* n_unknowns,
                         int64_t* n_floating, int64_t* near_pairs)
{
    if (!ctx) return BEM_ERR_ARG;
    if (n_panels) *n_panels = ctx->np;
    if (n_unknowns) *n_unknowns = ctx->nunk;
    if (n_floating) *n_floating = ctx->nfloat;
    if (near_pairs) *near_pairs = ctx->nnz;
    return BEM_OK;
}

extern "C" int bem_sync(bem_ctx* ctx)
{
    if (!ctx) return BEM_ERR_ARG;
    BEM_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
    int st = 0;
    BEM_CUDA_TRY(ctx, cudaMemcpy(&st, ctx->d_status, sizeof st, cudaMemcpyDeviceToHost));
    if (st != 0) {
        BEM_CUDA_TRY(ctx, cudaMemset(ctx->d_status, 0, sizeof(int)));
        return set_err(ctx, st, "device-side status %d", st);
    }
    return BEM_OK;
}

extern "C" int bem_destroy(bem_ctx* ctx)
{
    if (!ctx) return BEM_OK;
    cudaStreamSynchronize(ctx->stream);
    free_ctx(ctx);
    return BEM_OK;
}

// Tuner of the FP32 regular-pair kernel's shape: the variant (scalar, 2, 3 or 4 packed
// target pairs per thread) and the CTA slots per SM that the triangle-slice count
// aims at.  Each candidate is timed on the mesh's own mixed matvec (one warm-up, then
// CUDA events on the context's stream) and the fastest is kept.  The choice is kept
// in a process-wide table keyed by (device, size bucket floor(2 log2 N), far_order); later
// contexts of the same device and bucket take it from there without timing.
// params.far32_variant != 0 fixes the variant (slots 4); meshes below 4,096
// triangles take (2, 4) untimed.  The work counters are cleared afterwards.
namespace {
struct TuneChoice {
    int tp, slots;
};
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, TuneChoice> g_tune_table;  // (device, bucket, g)
}  // namespace

static int tune_far32(bem_ctx* c)
{
    const int bucket = (int)std::floor(2.0 * std::log2((double)std::max<int64_t>(c->np, 1)));
    bem_tuning& T = c->tune;
    T = bem_tuning{};
    T.bucket = bucket;
    if (c->prm.far32_variant != 0) {
        c->far32_tp = c->prm.far32_variant;
        c->far_slots = 4;
        T.source = 0;
    } else if (c->np < 4096) {
        c->far32_tp = 2;
        c->far_slots = 4;
        T.source = 0;
    } else {
        bool cached = false;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune_table.find(std::make_tuple(c->device, bucket, c->g));
            if (it != g_tune_table.end()) {
                c->far32_tp = it->second.tp;
                c->far_slots = it->second.slots;
                cached = true;
            }
        }
        if (cached) {
            T.source = 2;
        } else {
            cudaStream_t s = c->stream;
            cudaEvent_t e0, e1;
            BEM_CUDA_TRY(c, cudaEventCreate(&e0));
            BEM_CUDA_TRY(c, cudaEventCreate(&e1));
            std::vector<double> ones(c->nunk, 1.0);
            BEM_CUDA_TRY(c, cudaMemcpyAsync(c->zvec, ones.data(), c->nunk * sizeof(double),
                                            cudaMemcpyHostToDevice, s));
            float best = 3e38f;
            TuneChoice pick{2, 4};
            int k = 0;
            for (int tp : {1, 2, 3, 4}) {
                for (int sl : {2, 4, 8}) {
                    c->far32_tp = tp;
                    c->far_slots = sl;
                    int rc = matvec_impl(c, BEM_MIXED, 1, c->zvec, c->wvec);  // warm-up
                    if (!rc) {
                        cudaEventRecord(e0, s);
                        rc = matvec_impl(c, BEM_MIXED, 1, c->zvec, c->wvec);
                        cudaEventRecord(e1, s);
                    }
                    float ms = 3e38f;
                    if (!rc && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
                    if (rc) {
                        cudaEventDestroy(e0);
                        cudaEventDestroy(e1);
                        return rc;
                    }
                    T.cand_variant[k] = tp;
                    T.cand_slots[k] = sl;
                    T.cand_ms[k] = ms;
                    ++k;
                    if (ms < best) {
                        best = ms;
                        pick = {tp, sl};
                    }
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            T.n_candidates = k;
            T.source = 1;
            c->far32_tp = pick.tp;
            c->far_slots = pick.slots;
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tune_table[std::make_tuple(c->device, bucket, c->g)] = pick;
        }
    }
    T.far32_variant = c->far32_tp;
    T.far32_slots = c->far_slots;
    timing_drain(c);
    c->phi_tile_targets = far_phi_tile_targets(c);
    c->cnt = bem_counters{};
    c->cnt.far32_variant = c->far32_tp;
    BEM_CUDA_TRY(c, cudaMemsetAsync(c->d_near_count, 0, 4 * sizeof(unsigned long long), c->stream));
    BEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return BEM_OK;
}

extern "C" int bem_get_tuning(const bem_ctx* c, bem_tuning* out)
{
    if (!c || !out) return BEM_ERR_ARG;
    *out = c->tune;
    return BEM_OK;
}

extern "C" void bem_clear_tuning_table(void)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_table.clear();
}

static int create_impl(bem_ctx* c, const bem_mesh* mesh)
{
    const int64_t np = c->np, nv = c->nv;
    cudaStream_t s = c->stream;
    int rc;
    // quadrature rule (host) -> constant memory
    std::vector<double> u, wu, v, wv;
    host_gauss_rule(c->g, 1, u, wu);
    host_gauss_rule(c->g, 0, v, wv);
    if ((int)u.size() != c->g || (int)v.size() != c->g)
        return set_err(c, BEM_ERR_ARG, "quadrature rule of order %d could not be generated", c->g);
    c->h_rule_u = u; c->h_rule_wu = wu; c->h_rule_v = v; c->h_rule_wv = wv;
    BEM_CUDA_TRY(c, cudaMemcpyToSymbolAsync(c_rule_u, u.data(), c->g * sizeof(double), 0, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyToSymbolAsync(c_rule_wu, wu.data(), c->g * sizeof(double), 0, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyToSymbolAsync(c_rule_v, v.data(), c->g * sizeof(double), 0, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyToSymbolAsync(c_rule_wv, wv.data(), c->g * sizeof(double), 0, cudaMemcpyHostToDevice, s));

    const int Q = c->Q;
    if ((rc = dalloc(c, &c->X, 3 * nv)) || (rc = dalloc(c, &c->tri, 3 * np)) ||
        (rc = dalloc(c, &c->geo, GEO_STRIDE * np)) || (rc = dalloc(c, &c->hdr32, np)) ||
        (rc = dalloc(c, &c->hdr64, np)) || (rc = dalloc(c, &c->node32, Q * np)) ||
        (rc = dalloc(c, &c->node64, Q * np)) || (rc = dalloc(c, &c->tgt32, np)) ||
        (rc = dalloc(c, &c->tgt64, np)) || (rc = dalloc(c, &c->d_status, 1)) ||
        (rc = dalloc(c, &c->d_line_next, 1)) ||
        (rc = dalloc(c, &c->node_lo32, Q * np)) || (rc = dalloc(c, &c->tgt_lo32, np)) ||
        (rc = dalloc(c, &c->qnode, Q * np)) || (rc = dalloc(c, &c->chunk_sph, (np + 31) / 32)))
        return rc;
    BEM_CUDA_TRY(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(c->X, mesh->X, 3 * nv * sizeof(double), cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(c->tri, mesh->tri, 3 * np * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    k_panels<<<(unsigned)((np + 127) / 128), 128, 0, s>>>(np, c->g, c->prm.eta, c->X, c->tri, c->geo,
                                                          c->hdr32, c->hdr64, c->node32, c->node64,
                                                          c->tgt32, c->tgt64, c->node_lo32,
                                                          c->tgt_lo32, c->d_status);
    BEM_LAUNCH_CHECK(c);
    k_chunk_spheres<<<(unsigned)(((np + 31) / 32 + 127) / 128), 128, 0, s>>>(np, c->geo, c->chunk_sph);
    BEM_LAUNCH_CHECK(c);
    int st = 0;
    BEM_CUDA_TRY(c, cudaMemcpyAsync(&st, c->d_status, sizeof st, cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(c, cudaStreamSynchronize(s));
    if (st != 0) return set_err(c, BEM_ERR_DEGENERATE, "a triangle has zero area");

    // near pairs of the collocation points
    int32_t* d_count = nullptr;
    if ((rc = dalloc(c, &d_count, np)) || (rc = dalloc(c, &c->near_ptr, np + 1))) {
        if (d_count) cudaFree(d_count);
        return rc;
    }
    const unsigned wblocks = (unsigned)((np * 32 + 255) / 256);
    k_near_rows<<<wblocks, 256, 0, s>>>(np, 0, c->tgt32, c->tgt64, c->hdr32, c->hdr64, d_count,
                                         nullptr, nullptr, nullptr);
    std::vector<int32_t> cnt(np);
    std::vector<int64_t> ptr(np + 1);
    cudaError_t e = cudaMemcpyAsync(cnt.data(), d_count, np * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_count);
    if (e != cudaSuccess) return set_err(c, BEM_ERR_CUDA, "near count: %s", cudaGetErrorString(e));
    ptr[0] = 0;
    for (int64_t i = 0; i < np; ++i) ptr[i + 1] = ptr[i] + cnt[i];
    c->nnz = ptr[np];
    if ((rc = dalloc(c, &c->near_col, c->nnz)) || (rc = dalloc(c, &c->near_val, c->nnz)) ||
        (rc = dalloc(c, &c->near_flag, c->nnz)))
        return rc;
    BEM_CUDA_TRY(c, cudaMemcpyAsync(c->near_ptr, ptr.data(), (np + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    k_near_rows<<<wblocks, 256, 0, s>>>(np, 1, c->tgt32, c->tgt64, c->hdr32, c->hdr64, nullptr,
                                         c->near_ptr, c->near_col, c->near_flag);
    BEM_LAUNCH_CHECK(c);
    {
        // near pairs per precision, for the work counters
        std::vector<uint8_t> fl(c->nnz);
        BEM_CUDA_TRY(c, cudaMemcpyAsync(fl.data(), c->near_flag, c->nnz, cudaMemcpyDeviceToHost, s));
        BEM_CUDA_TRY(c, cudaStreamSynchronize(s));
        for (uint8_t f : fl) {
            c->nnz_prec[BEM_MIXED] += (f & 1) ? 1 : 0;
            c->nnz_prec[BEM_FP64] += (f & 2) ? 1 : 0;
            c->nnz_prec[kPrecDF] += (f & 1) ? 1 : 0;  // masked like FP32
        }
    }
    if ((rc = dalloc(c, &c->d_near_count, 4))) return rc;
    BEM_CUDA_TRY(c, cudaMemsetAsync(c->d_near_count, 0, 4 * sizeof(unsigned long long), s));
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
    BEM_LAUNCH_CHECK(c);
    if ((rc = dalloc(c, &c->near_val_df, c->nnz))) return rc;
    k_near_values<<<(unsigned)np, 64, 0, s>>>(np, Q, c->near_ptr, c->near_col, c->near_flag, c->geo,
                                               c->node64, c->near_val, c->near_val_df);
    BEM_LAUNCH_CHECK(c);

    // rows
    const int nreg = (int)c->regions.size();
    std::vector<int32_t> kind(np), aux(np);
    std::vector<double> ra(np, 0.0), rb(np, 0.0), rw(np, 0.0), rs(np, 0.0), V0(nreg, 0.0);
    std::vector<double> area_f(c->nfloat, 0.0);
    std::vector<std::vector<int32_t>> frows(c->nfloat);
    std::vector<double> h_area(np);
    {
        // areas are needed on the host for the neutrality weights
        std::vector<double> g(GEO_STRIDE * np);
        BEM_CUDA_TRY(c, cudaMemcpyAsync(g.data(), c->geo, g.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        BEM_CUDA_TRY(c, cudaStreamSynchronize(s));
        for (int64_t i = 0; i < np; ++i) h_area[i] = g[GEO_STRIDE * i + GEO_AREA];
    }
    for (int r = 0; r < nreg; ++r) V0[r] = c->regions[r].kind == BEM_CONDUCTOR ? c->regions[r].V0 : 0.0;
    // A sheet's rows are those of a floating conductor; only its neutrality
    // summand differs (Eq. sheets): the closed body's is A_i eps+ (u_i/2 + (K'u)_i),
    // the sheet's A_i ((eps+ + eps-)/2 u_i + (eps+ - eps-)(K'u)_i), both over area_f.
    // Both are written rw_i (u_i/2 + (K'u)_i) + rs_i u_i, with
    // rw_i = A_i (eps+ - eps-) / area_f and rs_i = A_i eps- / area_f, where a
    // closed body has eps- = 0 (no displacement field inside a conductor).
    for (int64_t i = 0; i < np; ++i) {
        const bem_region& R = c->regions[c->h_region[i]];
        const bool fl = R.kind == BEM_FLOATING || R.kind == BEM_SHEET;
        kind[i] = fl ? BEM_FLOATING : R.kind;
        aux[i] = fl ? R.floating_id : c->h_region[i];
        if (R.kind == BEM_DIELECTRIC) {
            ra[i] = 0.5 * (R.eps_plus + R.eps_minus);
            rb[i] = R.eps_plus - R.eps_minus;
        } else if (fl) {
            area_f[R.floating_id] += h_area[i];
            frows[R.floating_id].push_back((int32_t)i);
        }
    }
    for (int64_t i = 0; i < np; ++i) {
        const bem_region& R = c->regions[c->h_region[i]];
        if (R.kind == BEM_FLOATING) rw[i] = h_area[i] * R.eps_plus / area_f[R.floating_id];
        if (R.kind == BEM_SHEET) {
            rw[i] = h_area[i] * (R.eps_plus - R.eps_minus) / area_f[R.floating_id];
            rs[i] = h_area[i] * R.eps_minus / area_f[R.floating_id];
        }
    }
    std::vector<int32_t> fr, fo(c->nfloat + 1, 0);
    for (int f = 0; f < c->nfloat; ++f) {
        fr.insert(fr.end(), frows[f].begin(), frows[f].end());
        fo[f + 1] = (int32_t)fr.size();
    }
    if ((rc = dalloc(c, &c->row_kind, np)) || (rc = dalloc(c, &c->row_aux, np)) ||
        (rc = dalloc(c, &c->row_a, np)) || (rc = dalloc(c, &c->row_b, np)) ||
        (rc = dalloc(c, &c->row_w, np)) || (rc = dalloc(c, &c->row_s, np)) ||
        (rc = dalloc(c, &c->region_V0, nreg)) ||
        (rc = dalloc(c, &c->float_rows, fr.size())) || (rc = dalloc(c, &c->float_off, fo.size())) ||
        (rc = dalloc(c, &c->jinv, c->nunk)))
        return rc;
    BEM_CUDA_TRY(c, cudaMemcpyAsync(c->row_kind, kind.data(), np * 4, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(c->row_aux, aux.data(), np * 4, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(c->row_a, ra.data(), np * 8, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(c->row_b, rb.data(), np * 8, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(c->row_w, rw.data(), np * 8, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(c->row_s, rs.data(), np * 8, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(c->region_V0, V0.data(), nreg * 8, cudaMemcpyHostToDevice, s));
    {
        // bodies whose surface ends a field line; a thin sheet has no inside
        std::vector<int32_t> elec(nreg);
        for (int r = 0; r < nreg; ++r)
            elec[r] = (c->regions[r].kind == BEM_CONDUCTOR || c->regions[r].kind == BEM_FLOATING) ? 1 : 0;
        if ((rc = dalloc(c, &c->d_region, np)) || (rc = dalloc(c, &c->d_electrode, nreg)) ||
            (rc = dalloc(c, &c->nrm32, np)) || (rc = dalloc(c, &c->u32, np)))
            return rc;
        BEM_CUDA_TRY(c, cudaMemcpyAsync(c->d_region, c->h_region.data(), np * 4, cudaMemcpyHostToDevice, s));
        BEM_CUDA_TRY(c, cudaMemcpyAsync(c->d_electrode, elec.data(), nreg * 4, cudaMemcpyHostToDevice, s));
        k_nrm32<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(np, c->geo, c->d_region, c->nrm32);
        BEM_LAUNCH_CHECK(c);
        BEM_CUDA_TRY(c, cudaStreamSynchronize(s));
    }
    if (!fr.empty())
        BEM_CUDA_TRY(c, cudaMemcpyAsync(c->float_rows, fr.data(), fr.size() * 4, cudaMemcpyHostToDevice, s));
    BEM_CUDA_TRY(c, cudaMemcpyAsync(c->float_off, fo.data(), fo.size() * 4, cudaMemcpyHostToDevice, s));
    k_jacobi<<<(unsigned)((c->nunk + 255) / 256), 256, 0, s>>>(np, c->nunk, c->row_kind, c->row_a,
                                                               c->near_ptr, c->near_col,
                                                               c->near_val, c->jinv);
    BEM_LAUNCH_CHECK(c);

    // workspace: far partials for the largest launch
    const int64_t Mmax = std::max<int64_t>(np, c->prm.max_points);
    size_t need = 0;
    const int tp_default = c->far32_tp, slots_default = c->far_slots;
    for (int tp : {1, 2, 3, 4}) {  // every FP32 kernel shape the tuner may pick
        for (int sl : {2, 4, 8}) {
            c->far32_tp = tp;
            c->far_slots = sl;
            for (int prec = 0; prec < 3; ++prec) {
                for (int64_t M : {np, (int64_t)c->prm.max_points}) {
                    const size_t n = (size_t)far_splits(c, prec, M) * (size_t)M * 4 * kMaxRhs;
                    need = std::max(need, n);
                }
            }
        }
    }
    c->far32_tp = tp_default;
    c->far_slots = slots_default;
    (void)Mmax;
    c->part_cap = need;
    c->m = c->prm.gmres_restart;
    const int64_t n = c->nunk;
    if ((rc = dalloc(c, &c->part, need)) || (rc = dalloc(c, &c->field, (size_t)kMaxRhs * np * 4)) ||
        (rc = dalloc(c, &c->neut, (size_t)kMaxRhs * np)) ||
        (rc = dalloc(c, &c->V, (size_t)(c->m + 1) * n)) || (rc = dalloc(c, &c->wvec, n)) ||
        (rc = dalloc(c, &c->zvec, n)) || (rc = dalloc(c, &c->rvec, n)) ||
        (rc = dalloc(c, &c->bvec, n)) || (rc = dalloc(c, &c->dvec, n)) ||
        (rc = dalloc(c, &c->ivec, n)) ||
        (rc = dalloc(c, &c->hcol, 2 * (c->m + 2))) ||
        (rc = dalloc(c, &c->ord_pts, 3 * (size_t)c->prm.max_points)) ||
        (rc = dalloc(c, &c->ord_perm, (size_t)c->prm.max_points)) ||
        (rc = dalloc(c, &c->ord_cell, (size_t)c->prm.max_points)) ||
        (rc = dalloc(c, &c->ord_hist, (size_t)order_hist_len(c->prm.max_points))) ||
        (rc = dalloc(c, &c->ord_box, (size_t)order_box_len())))
        return rc;
    if (cudaMallocHost((void**)&c->hcol_host, 2 * (c->m + 2) * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        c->hcol_host = nullptr;
        return set_err(c, BEM_ERR_NOMEM, "cudaMallocHost failed");
    }
    BEM_CUDA_TRY(c, cudaStreamSynchronize(s));
    if ((rc = tune_far32(c))) return rc;
    if ((rc = adjoint_workspace_create(c))) return rc;
    return BEM_OK;
}

extern "C" int bem_create(bem_ctx** out, const bem_mesh* mesh, const bem_params* params, void* stream)
{
    if (!out) return set_err(nullptr, BEM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!mesh || !mesh->X || !mesh->tri || !mesh->region || !mesh->regions)
        return set_err(nullptr, BEM_ERR_ARG, "mesh or one of its arrays is NULL");
    if (mesh->nv < 3 || mesh->np < 1 || mesh->nregions < 1 || mesh->np > (int64_t)1 << 30)
        return set_err(nullptr, BEM_ERR_ARG, "bad sizes nv=%lld np=%lld nregions=%d",
                       (long long)mesh->nv, (long long)mesh->np, mesh->nregions);
    bem_params prm;
    if (params)
        prm = *params;
    else
        bem_default_params(&prm);
    if (!(prm.eta >= 1.0) || prm.far_order < 1 || prm.far_order > kMaxOrder ||
        prm.gmres_restart < 1 || prm.gmres_restart > 1000 || prm.max_iters < 1 ||
        prm.adjoint_lines < 0 || prm.adjoint_checkpoint < 1 || prm.trace_cluster < 0 || prm.trace_cluster > 8 ||
        prm.max_refine < 1 || prm.max_points < 1 || prm.max_points > INT32_MAX ||
        (prm.residual != BEM_RESIDUAL_DF && prm.residual != BEM_RESIDUAL_FP64 &&
         prm.residual != BEM_RESIDUAL_DF_UPDATE) ||
        (prm.far32_variant != 0 && (prm.far32_variant < 1 || prm.far32_variant > 4)))
        return set_err(nullptr, BEM_ERR_ARG, "bad parameters (need eta >= 1, 1 <= far_order <= %d)",
                       kMaxOrder);
    for (int64_t i = 0; i < 3 * mesh->np; ++i)
        if (mesh->tri[i] < 0 || mesh->tri[i] >= mesh->nv)
            return set_err(nullptr, BEM_ERR_ARG, "vertex index out of range in triangle %lld",
                           (long long)(i / 3));
    int nfloat = 0;
    for (int r = 0; r < mesh->nregions; ++r) {
        const bem_region& R = mesh->regions[r];
        if (R.kind < BEM_CONDUCTOR || R.kind > BEM_SHEET)
            return set_err(nullptr, BEM_ERR_ARG, "region %d: unknown kind %d", r, R.kind);
        if (R.kind == BEM_FLOATING || R.kind == BEM_SHEET) {
            if (R.floating_id < 0 || R.floating_id >= mesh->nregions)
                return set_err(nullptr, BEM_ERR_ARG, "region %d: bad floating_id", r);
            nfloat = std::max(nfloat, R.floating_id + 1);
            if (!(R.eps_plus > 0.0)) return set_err(nullptr, BEM_ERR_ARG, "region %d: eps_plus <= 0", r);
        }
        if (R.kind == BEM_SHEET && !(R.eps_minus >= 0.0))
            return set_err(nullptr, BEM_ERR_ARG, "region %d: sheet eps_minus < 0", r);
        if (R.kind == BEM_DIELECTRIC && (!(R.eps_plus > 0.0) || !(R.eps_minus > 0.0)))
            return set_err(nullptr, BEM_ERR_ARG, "region %d: permittivities must be > 0", r);
    }
    std::vector<int> seen(nfloat, 0);
    for (int64_t i = 0; i < mesh->np; ++i) {
        const int r = mesh->region[i];
        if (r < 0 || r >= mesh->nregions)
            return set_err(nullptr, BEM_ERR_ARG, "region index out of range at triangle %lld", (long long)i);
        if (mesh->regions[r].kind == BEM_FLOATING || mesh->regions[r].kind == BEM_SHEET)
            seen[mesh->regions[r].floating_id] = 1;
    }
    for (int f = 0; f < nfloat; ++f)
        if (!seen[f]) return set_err(nullptr, BEM_ERR_ARG, "floating id %d has no triangles", f);

    bem_ctx* c = new (std::nothrow) bem_ctx();
    if (!c) return set_err(nullptr, BEM_ERR_NOMEM, "host allocation failed");
    c->stream = (cudaStream_t)stream;
    c->prm = prm;
    c->nv = mesh->nv;
    c->np = mesh->np;
    c->nfloat = nfloat;
    c->nunk = mesh->np + nfloat;
    c->g = prm.far_order;
    c->Q = prm.far_order * prm.far_order;
    c->regions.assign(mesh->regions, mesh->regions + mesh->nregions);
    c->h_region.assign(mesh->region, mesh->region + mesh->np);
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
        set_err(nullptr, BEM_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
        cudaGetLastError();
        delete c;
        return BEM_ERR_CUDA;
    }
    const int rc = create_impl(c, mesh);
    if (rc != BEM_OK) {
        g_create_err = c->err;
        free_ctx(c);
        return rc;
    }
    *out = c;
    return BEM_OK;
}

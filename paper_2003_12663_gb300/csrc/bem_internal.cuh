// bem_internal.cuh -- context layout, device helpers and launchers shared by the
// translation units of libbem.so.  Nothing here is part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "bem.h"

// ---------------------------------------------------------------- panel record
// Per triangle, FP64, 24 doubles (192 B, 16-B aligned):
//   a[3] b[3] c[3]  vertices (CCW about n)
//   n[3]            unit normal
//   area
//   ctr[3]          centroid (collocation point, Sec. 3)
//   cc[3]           circumcentre (classification, Sec. 4)
//   R               circumradius
//   etaR            eta * R
//   pad[2]
enum { GEO_A = 0, GEO_B = 3, GEO_C = 6, GEO_N = 9, GEO_AREA = 12, GEO_CTR = 13, GEO_CC = 16,
       GEO_R = 19, GEO_ETAR = 20, GEO_STRIDE = 24 };

constexpr int kMaxOrder = 6;          // largest far_order g
constexpr int kMaxRhs = 4;            // right-hand sides per matvec launch
constexpr int kPrecDF = BEM_DF;       // regular pairs in double-FP32 arithmetic
constexpr double kInv4Pi = 0.07957747154594767;  // 1/(4 pi)

struct AdjWork;  // adjoint.cu: the workspace of bem_adjoint
struct P1Data;   // p1.cu: a context of curved six-node triangles with P1 densities

struct bem_ctx {
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    bem_params prm{};
    int64_t nv = 0, np = 0, nunk = 0;
    int nfloat = 0;
    int g = 3, Q = 9;
    std::vector<bem_region> regions;
    std::vector<int32_t> h_region;
    std::vector<double> h_rule_u, h_rule_wu, h_rule_v, h_rule_wv;  // the far rule, host copy

    // geometry
    double* X = nullptr;        // [nv][3]
    int32_t* tri = nullptr;     // [np][3]
    double* geo = nullptr;      // [np][GEO_STRIDE]
    float4* hdr32 = nullptr;    // [np] (cc, (eta R)^2)    FP32
    double4* hdr64 = nullptr;   // [np] (cc, (eta R)^2)    FP64
    float4* node32 = nullptr;   // [np][Q] (y, w)          FP32
    double4* node64 = nullptr;  // [np][Q] (y, w)          FP64
    float4* node_lo32 = nullptr;  // [np][Q] node - node32 (low parts of the double-FP32 nodes)
    float4* qnode = nullptr;      // [np][Q] FP32 nodes with sigma folded into w (per call)
    float4* chunk_sph = nullptr;  // [np/32 rounded up] bounding sphere of 32 triangles' near zones
    int far32_tp = 2;             // FP32 kernel variant: 1 scalar, 2, 3 or 4 packed target pairs
    int far_slots = 4;            // CTA slots per SM the FP32 kernel's slice count aims at (tuned)
    bem_tuning tune{};            // what the tuner chose and measured
    int64_t phi_tile_targets = 0; // centroid targets in tiles of conductor rows only (packed variant)
    float4* nrm32 = nullptr;      // [np] (unit normal in FP32, region index as int bits): field lines
    float* u32 = nullptr;         // [np] density rounded to FP32 for the field-line integrator
    float4* tgt_lo32 = nullptr;   // [np] centroid - tgt32
    float4* tgt32 = nullptr;    // [np] centroids          FP32
    double4* tgt64 = nullptr;   // [np] centroids          FP64

    // rows (Eqs. Final1-Final4)
    int32_t* row_kind = nullptr;   // [np]
    int32_t* row_aux = nullptr;    // [np] floating id or region index of a conductor
    double* row_a = nullptr;       // [np] dielectric: (eps+ + eps-)/2
    double* row_b = nullptr;       // [np] dielectric: eps+ - eps-
    double* row_w = nullptr;       // [np] floating: A_i eps+ / area_f; sheet: A_i (eps+ - eps-) / area_f
    double* row_s = nullptr;       // [np] sheet: A_i eps- / area_f (0 elsewhere)
    double* region_V0 = nullptr;   // [nregions]
    int32_t* d_region = nullptr;   // [np] region of every triangle
    int32_t* d_electrode = nullptr;  // [nregions] 1 for conductor and floating regions (not sheets)
    int32_t* float_rows = nullptr; // rows of every floating body, grouped
    int32_t* float_off = nullptr;  // [nfloat+1]
    double* jinv = nullptr;        // [nunk] inverse Jacobi diagonal

    // near pairs of the collocation points (CSR over rows, columns ascending)
    int64_t nnz = 0;
    int64_t* near_ptr = nullptr;   // [np+1]
    int32_t* near_col = nullptr;   // [nnz]
    double4* near_val = nullptr;   // [nnz] exact (S, G) of the pair, G's normal part PV for i==j
    double4* near_val_df = nullptr;  // [nnz] what the double-FP32 pass adds (see k_near_values)
    int64_t* csc_ptr = nullptr;    // near pairs by column (built on the first transposed product)
    int32_t* csc_row = nullptr;
    int64_t* csc_ent = nullptr;    // index of the pair in the row-ordered arrays
    double4* tsrc64 = nullptr;     // [np] sources of the transposed product
    float4* tsrc32 = nullptr;
    uint8_t* near_flag = nullptr;  // [nnz] bit0: near in FP32 classification, bit1: in FP64

    // workspace
    double* part = nullptr;        // far partial sums
    size_t part_cap = 0;           // doubles
    double* field = nullptr;       // [kMaxRhs][np][4] reduced phi, E at the centroids
    double* neut = nullptr;        // [kMaxRhs][np] neutrality contributions
    double* pts_stage = nullptr;   // staging for host points (unused by device-pointer calls)
    // spatial order of one chunk of evaluation points (order.cu)
    double* ord_pts = nullptr;     // [max_points][3] the points in cell order
    int32_t* ord_perm = nullptr;   // [max_points] input index of each ordered point
    int32_t* ord_cell = nullptr;   // [max_points] cell of each input point
    int32_t* ord_hist = nullptr;   // [order_hist_len] per-block cell counts, then offsets
    float* ord_box = nullptr;      // [order_box_len] partial bounding boxes

    // solver workspace
    int m = 100;
    double* V = nullptr;           // [(m+1)][nunk] Krylov basis
    double* wvec = nullptr;        // [nunk]
    double* zvec = nullptr;        // [nunk]
    double* rvec = nullptr;        // [nunk]
    double* bvec = nullptr;        // [nunk]
    double* dvec = nullptr;        // [nunk]
    double* ivec = nullptr;        // [nunk]
    double* hcol = nullptr;        // [2(m+2)] device Hessenberg column scratch
    double* hcol_host = nullptr;   // pinned mirror
    int* d_status = nullptr;       // device-side status word
    unsigned long long* d_line_next = nullptr;  // line counter of the persistent tracer launches

    // work counters (bem_counters) and optional kernel timing
    bem_counters cnt{};
    int64_t nnz_prec[3] = {0, 0, 0};          // near pairs of the centroids per pass
    unsigned long long* d_near_count = nullptr;  // [4] near pairs met by the point kernels (FP64, FP32);
                                                 // chunks of k_far32p, of which all-regular
    std::vector<cudaEvent_t> ev0, ev1;        // timing pool: start / stop of far launches
    std::vector<int> ev_prec;
    size_t ev_used = 0;

    AdjWork* adj = nullptr;        // adjoint workspace (params.adjoint_lines > 0)
    // curved-triangle (P1) context: the regular-pair kernels take the density folded
    // into qnode / qnode64 per product, with a unit factor per triangle (ones)
    P1Data* p1 = nullptr;
    double4* qnode64 = nullptr;
    const double* ones = nullptr;

    std::string err;
};

// p1.cu: the curved-triangle path behind the generic calls
int p1_matvec_impl(bem_ctx* ctx, int precision, int nrhs, const double* x, double* y);
int p1_rhs(bem_ctx* ctx, int nrhs, const double* V0, double* b);
int p1_eval_field(bem_ctx* ctx, int precision, const double* u, int64_t M, const double* pts, double* phi,
                  double* E);
int p1_assemble(bem_ctx* ctx, int64_t row0, int64_t row1, int precision, double* A, int64_t lda);
void p1_free(bem_ctx* ctx);
// setup.cu: n-point Gauss-Legendre rule on [-1, 1]; bounding spheres of 32-triangle chunks
void gauss_legendre_pm1(int n, std::vector<double>& x, std::vector<double>& w);
__global__ void k_chunk_spheres(int64_t np, const double* __restrict__ geo, float4* __restrict__ sph);

// adjoint.cu: the adjoint workspace, allocated by bem_create and freed with the context
int adjoint_workspace_create(bem_ctx* ctx);
void adjoint_workspace_free(bem_ctx* ctx);

// timing of the regular-pair launches (setup.cu)
void timing_begin(bem_ctx* ctx, int precision);
void timing_end(bem_ctx* ctx);

// ---------------------------------------------------------------- error helpers
int set_err(bem_ctx* ctx, int code, const char* fmt, ...);
#define BEM_CUDA_TRY(ctx, call)                                                              \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return set_err((ctx), BEM_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)
// after every kernel launch: count it and report a launch error
#define BEM_LAUNCH_CHECK(ctx)                       \
    do {                                            \
        ++(ctx)->cnt.kernel_launches;               \
        BEM_CUDA_TRY(ctx, cudaGetLastError());      \
    } while (0)

// ---------------------------------------------------------------- device helpers
// The pair classification of Sec. 4, written once per precision with explicit
// rounding so that every kernel of that precision takes the same decision for
// the same (target, triangle): regular ("far") iff |x - cc|^2 > (eta R)^2.
__device__ __forceinline__ bool is_far32(float x, float y, float z, float4 h)
{
    const float dx = __fsub_rn(x, h.x), dy = __fsub_rn(y, h.y), dz = __fsub_rn(z, h.z);
    const float d2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    return d2 > h.w;
}

__device__ __forceinline__ bool is_far64(double x, double y, double z, double4 h)
{
    const double dx = __dsub_rn(x, h.x), dy = __dsub_rn(y, h.y), dz = __dsub_rn(z, h.z);
    const double d2 = __fma_rn(dz, dz, __fma_rn(dy, dy, __dmul_rn(dx, dx)));
    return d2 > h.w;
}

// Closed-form integrals of a uniform unit density over a flat triangle (FP64).
// For every edge p->q (unit tangent t, outward in-plane normal m = t x n) the
// line integral f = int_edge dl/|x-y| is taken in the form that avoids
// cancellation: with s0 = (p-x).t, s1 = (q-x).t, r0 = |p-x|, r1 = |q-x|,
// L = |q-p|,
//   s0 >= 0: f = log1p(L (s0+s1+r0+r1) / ((r0+r1)(r0+s0)))
//   s1 <= 0: f = log1p(L (r0+r1-s0-s1) / ((r0+r1)(r1-s1)))
//   else   : f = log((r1+s1)(r0-s0) / (d^2+h^2)),  d = (p-x).m, h = (x-a).n.
// With the signed solid angle Omega of the triangle seen from x (Van Oosterom &
// Strackee; negative on the side n points to):
//   4 pi S = sum d f + h Omega,   4 pi G = sum m f - Omega n.
// own != 0: x is this triangle's centroid, the normal part of G is its
// principal value (0) and h = 0.
__device__ __forceinline__ void tri_closed_form(const double* __restrict__ gp, double x,
                                                double y, double z, bool own, double& S,
                                                double& Gx, double& Gy, double& Gz)
{
    const double nx = gp[GEO_N], ny = gp[GEO_N + 1], nz = gp[GEO_N + 2];
    const double h = own ? 0.0 : (x - gp[GEO_A]) * nx + (y - gp[GEO_A + 1]) * ny + (z - gp[GEO_A + 2]) * nz;
    double sdf = 0.0, fx = 0.0, fy = 0.0, fz = 0.0;
    double ax[3], ay[3], az[3], al[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        ax[i] = gp[3 * i] - x;
        ay[i] = gp[3 * i + 1] - y;
        az[i] = gp[3 * i + 2] - z;
        al[i] = sqrt(ax[i] * ax[i] + ay[i] * ay[i] + az[i] * az[i]);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int k = (i + 1) % 3;
        const double ex = ax[k] - ax[i], ey = ay[k] - ay[i], ez = az[k] - az[i];
        const double L = sqrt(ex * ex + ey * ey + ez * ez);
        const double tx = ex / L, ty = ey / L, tz = ez / L;
        const double mx = ty * nz - tz * ny, my = tz * nx - tx * nz, mz = tx * ny - ty * nx;
        const double s0 = ax[i] * tx + ay[i] * ty + az[i] * tz;
        const double s1 = ax[k] * tx + ay[k] * ty + az[k] * tz;
        const double r0 = al[i], r1 = al[k];
        const double d = ax[i] * mx + ay[i] * my + az[i] * mz;
        double f;
        if (s0 >= 0.0)
            f = log1p(L * (s0 + s1 + r0 + r1) / ((r0 + r1) * (r0 + s0)));
        else if (s1 <= 0.0)
            f = log1p(L * (r0 + r1 - s0 - s1) / ((r0 + r1) * (r1 - s1)));
        else
            f = log((r1 + s1) * (r0 - s0) / (d * d + h * h));
        if (d != 0.0) sdf += d * f;
        fx += mx * f;
        fy += my * f;
        fz += mz * f;
    }
    double om = 0.0;
    if (!own) {
        const double det = ax[0] * (ay[1] * az[2] - az[1] * ay[2]) - ay[0] * (ax[1] * az[2] - az[1] * ax[2]) +
                           az[0] * (ax[1] * ay[2] - ay[1] * ax[2]);
        const double d01 = ax[0] * ax[1] + ay[0] * ay[1] + az[0] * az[1];
        const double d02 = ax[0] * ax[2] + ay[0] * ay[2] + az[0] * az[2];
        const double d12 = ax[1] * ax[2] + ay[1] * ay[2] + az[1] * az[2];
        const double den = al[0] * al[1] * al[2] + d01 * al[2] + d02 * al[1] + d12 * al[0];
        om = 2.0 * atan2(det, den);
    }
    S = kInv4Pi * (sdf + h * om);
    Gx = kInv4Pi * (fx - om * nx);
    Gy = kInv4Pi * (fy - om * ny);
    Gz = kInv4Pi * (fz - om * nz);
}

// ---------------------------------------------------------------- launchers
// far.cu: partial sums of sum_j u_j (S_j, G_j)(x_t) over regular pairs, one
// (split, target) record of 4 doubles per right-hand side.
struct FarTargets {
    const float4* t32;       // FP32 targets (x,y,z,-) or nullptr
    const float4* t32lo;     // low parts for the double-FP32 pass (centroid targets only)
    const double4* t64;      // FP64 targets (x,y,z,-) or nullptr
    const double* tpts;      // or raw double [M][3]
    int64_t M;
    const int32_t* phi_kind = nullptr;  // row kinds: tiles of conductor rows may skip E (matvec only)
};
int far_splits(const bem_ctx* ctx, int precision, int64_t M);
// centroid targets whose packed-kernel tile holds conductor rows only (0 for the scalar variant)
int64_t far_phi_tile_targets(const bem_ctx* ctx);
int launch_far(bem_ctx* ctx, int precision, const FarTargets& T, const double* u, int nrhs,
               int64_t ustride, int splits, double* part);

// field.cu
constexpr int64_t kOrderMin = 4096;  // bem_eval_field orders chunks of at least this many points
int64_t order_hist_len(int64_t max_points);
int64_t order_box_len();
int order_points(bem_ctx* c, int64_t M, const double* pts, double* spts, int32_t* perm);
int launch_points_near(bem_ctx* ctx, int precision, int64_t M, const double* pts, const double* u,
                       const double* part, int splits, double* phi, double* E);
// need_E: also fill ctx->field with E at the conductor rows (otherwise their regular
// pairs may be summed for phi alone, which is all their row equation uses)
int matvec_impl(bem_ctx* ctx, int precision, int nrhs, const double* x, double* y, bool need_E = false);
// adjoint.cu: y = A^T v (one right-hand side)
int matvecT_impl(bem_ctx* ctx, int precision, const double* v, double* y);

// setup.cu
void host_gauss_rule(int n, int weight_power, std::vector<double>& x, std::vector<double>& w);

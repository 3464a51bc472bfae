// solver.cu -- restarted GMRES with right Jacobi scaling (Sec. 3: Krylov methods
// need only matrix-vector products; Sec. 5: GMRES with a diagonal
// preconditioner) on the matrix-free matvec, and, for BEM_MIXED, an iterative
// refinement whose residual b - A u is formed with the FP64 form's operator (in
// double-FP32 arithmetic, or with the FP64 kernel); by default only the first
// residual of a solve is formed so, and the later ones are updated with the mixed
// product of each (small) correction.
//
// The Krylov basis, the orthogonalisation (classical Gram-Schmidt applied
// twice) and all vectors stay on the device in FP64; only the new Hessenberg
// column (at most m+2 numbers) comes back to the host each iteration, where
// the Givens rotations and the small triangular solve run.
#include <cmath>
#include <vector>

#include "bem_internal.cuh"

namespace {

constexpr int kDotThreads = 256;

// out[k] = <V_k, w> for k < nv (one block per vector, fixed-order reduction)
__global__ void k_dots(const double* __restrict__ V, int64_t ld, int nv, const double* __restrict__ w,
                       int64_t n, double* __restrict__ out)
{
    __shared__ double sh[kDotThreads];
    const int k = blockIdx.x;
    if (k >= nv) return;
    const double* v = V + (int64_t)k * ld;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kDotThreads) s = fma(v[i], w[i], s);
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = kDotThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[k] = sh[0];
}

// w -= sum_k V_k h_k ;  if acc: hsum[k] += h[k] (done by thread 0 of block 0)
__global__ void k_subtract(double* __restrict__ w, const double* __restrict__ V, int64_t ld, int nv,
                           const double* __restrict__ h, int64_t n, double* __restrict__ hsum)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (hsum && blockIdx.x == 0)
        for (int k = threadIdx.x; k < nv; k += blockDim.x) hsum[k] += h[k];
    if (i >= n) return;
    double s = w[i];
    for (int k = 0; k < nv; ++k) s = fma(-V[(int64_t)k * ld + i], h[k], s);
    w[i] = s;
}

// y = a * x  with a = 1/nrm[0] (nrm on device)
__global__ void k_scale_inv(double* __restrict__ y, const double* __restrict__ x,
                            const double* __restrict__ nrm, int64_t n)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double s = sqrt(nrm[0]);
    y[i] = s > 0.0 ? x[i] / s : 0.0;
}

__global__ void k_mul(double* __restrict__ z, const double* __restrict__ a,
                      const double* __restrict__ b, int64_t n)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) z[i] = a[i] * b[i];
}

// x += jinv .* (V y)
__global__ void k_update(double* __restrict__ x, const double* __restrict__ jinv,
                         const double* __restrict__ V, int64_t ld, int nv,
                         const double* __restrict__ y, int64_t n)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int k = 0; k < nv; ++k) s = fma(V[(int64_t)k * ld + i], y[k], s);
    x[i] = fma(jinv[i], s, x[i]);
}

// r = b - r  (r holds A x on entry)
__global__ void k_resid(double* __restrict__ r, const double* __restrict__ b, int64_t n)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) r[i] = b[i] - r[i];
}

__global__ void k_axpy(double* __restrict__ y, const double* __restrict__ x, int64_t n)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] += x[i];
}

__global__ void k_sub(double* __restrict__ y, const double* __restrict__ x, int64_t n)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] -= x[i];
}

inline unsigned nb(int64_t n) { return (unsigned)((n + 255) / 256); }

int norm2(bem_ctx* c, const double* x, double* out_host)
{
    k_dots<<<1, kDotThreads, 0, c->stream>>>(x, 0, 1, x, c->nunk, c->hcol);
    BEM_LAUNCH_CHECK(c);
    BEM_CUDA_TRY(c, cudaMemcpyAsync(c->hcol_host, c->hcol, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    BEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    *out_host = std::sqrt(c->hcol_host[0]);
    return BEM_OK;
}

// y = A x or A^T x
int apply(bem_ctx* c, int precision, bool transpose, const double* x, double* y)
{
    return transpose ? matvecT_impl(c, precision, x, y) : matvec_impl(c, precision, 1, x, y);
}

// r = b - A x (or b - A^T x) with the given precision
int residual(bem_ctx* c, int precision, const double* b, const double* x, double* r, bool transpose = false)
{
    int rc = apply(c, precision, transpose, x, r);
    if (rc) return rc;
    k_resid<<<nb(c->nunk), 256, 0, c->stream>>>(r, b, c->nunk);
    BEM_LAUNCH_CHECK(c);
    return BEM_OK;
}

// GMRES(m) on A x = b, x in/out (device), stop at ||b - A x|| <= tol_abs.
// Uses c->rvec, wvec, zvec, V.  iters is incremented per Arnoldi step.
int gmres(bem_ctx* c, int precision, const double* b, double* x, bool x_zero, double tol_abs,
          int max_iters, int* iters, double* res_out, bool transpose = false)
{
    const int64_t n = c->nunk;
    const int m = c->m;
    cudaStream_t s = c->stream;
    double* r = c->rvec;
    double* w = c->wvec;
    double* z = c->zvec;
    double* hd = c->hcol;        // device: [0..m+1] h of this column, [m+2..] scratch
    double* hh = c->hcol_host;
    int rc;
    if (x_zero) {
        BEM_CUDA_TRY(c, cudaMemcpyAsync(r, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else if ((rc = residual(c, precision, b, x, r, transpose))) {
        return rc;
    }
    double beta;
    if ((rc = norm2(c, r, &beta))) return rc;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
    while (true) {
        *res_out = beta;
        if (beta <= tol_abs) return BEM_OK;
        if (*iters >= max_iters) return BEM_ERR_NOT_CONVERGED;
        // v_0 = r / beta
        BEM_CUDA_TRY(c, cudaMemsetAsync(hd, 0, sizeof(double), s));
        hh[0] = beta * beta;
        BEM_CUDA_TRY(c, cudaMemcpyAsync(hd, hh, sizeof(double), cudaMemcpyHostToDevice, s));
        k_scale_inv<<<nb(n), 256, 0, s>>>(c->V, r, hd, n);
        BEM_LAUNCH_CHECK(c);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int j = 0;
        double res = beta;
        for (; j < m && *iters < max_iters; ++j) {
            double* vj = c->V + (int64_t)j * n;
            k_mul<<<nb(n), 256, 0, s>>>(z, c->jinv, vj, n);
            BEM_LAUNCH_CHECK(c);
            if ((rc = apply(c, precision, transpose, z, w))) return rc;
            // classical Gram-Schmidt, twice; h accumulates in hd[0..j]
            double* hsum = hd;
            double* htmp = hd + (m + 2);
            BEM_CUDA_TRY(c, cudaMemsetAsync(hsum, 0, (j + 1) * sizeof(double), s));
            for (int pass = 0; pass < 2; ++pass) {
                k_dots<<<j + 1, kDotThreads, 0, s>>>(c->V, n, j + 1, w, n, htmp);
                BEM_LAUNCH_CHECK(c);
                k_subtract<<<nb(n), 256, 0, s>>>(w, c->V, n, j + 1, htmp, n, hsum);
                BEM_LAUNCH_CHECK(c);
            }
            k_dots<<<1, kDotThreads, 0, s>>>(w, 0, 1, w, n, hsum + j + 1);
            BEM_LAUNCH_CHECK(c);
            k_scale_inv<<<nb(n), 256, 0, s>>>(c->V + (int64_t)(j + 1) * n, w, hsum + j + 1, n);
            BEM_LAUNCH_CHECK(c);
            BEM_CUDA_TRY(c, cudaMemcpyAsync(hh, hsum, (j + 2) * sizeof(double), cudaMemcpyDeviceToHost, s));
            BEM_CUDA_TRY(c, cudaStreamSynchronize(s));
            ++*iters;
            ++c->cnt.gmres_iters;
            double* Hj = &H[(size_t)j * (m + 1)];  // column j
            for (int k = 0; k <= j; ++k) Hj[k] = hh[k];
            Hj[j + 1] = std::sqrt(std::max(hh[j + 1], 0.0));
            for (int k = 0; k < j; ++k) {  // previous rotations
                const double t = cs[k] * Hj[k] + sn[k] * Hj[k + 1];
                Hj[k + 1] = -sn[k] * Hj[k] + cs[k] * Hj[k + 1];
                Hj[k] = t;
            }
            const double den = std::hypot(Hj[j], Hj[j + 1]);
            cs[j] = den > 0.0 ? Hj[j] / den : 1.0;
            sn[j] = den > 0.0 ? Hj[j + 1] / den : 0.0;
            Hj[j] = den;
            Hj[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            res = std::fabs(g[j + 1]);
            if (res <= tol_abs || den == 0.0) { ++j; break; }
        }
        // y = H^{-1} g  (upper triangular j x j)
        for (int k = j - 1; k >= 0; --k) {
            double t = g[k];
            for (int l = k + 1; l < j; ++l) t -= H[(size_t)l * (m + 1) + k] * y[l];
            const double d = H[(size_t)k * (m + 1) + k];
            y[k] = d != 0.0 ? t / d : 0.0;
        }
        BEM_CUDA_TRY(c, cudaMemcpyAsync(hd, y.data(), j * sizeof(double), cudaMemcpyHostToDevice, s));
        k_update<<<nb(n), 256, 0, s>>>(x, c->jinv, c->V, n, j, hd, n);
        BEM_LAUNCH_CHECK(c);
        // true residual of the restart
        if ((rc = residual(c, precision, b, x, r, transpose))) return rc;
        if ((rc = norm2(c, r, &beta))) return rc;
    }
}

}  // namespace

// A^T x = rhs by GMRES with the same right Jacobi scaling (diag(A^T) = diag(A));
// x starts from 0.  Used by the adjoint.
int solve_transpose(bem_ctx* c, int precision, const double* rhs, double* x, double tol, int* iters,
                    double* relres)
{
    BEM_CUDA_TRY(c, cudaMemsetAsync(x, 0, c->nunk * sizeof(double), c->stream));
    double bnorm;
    if (int rc = norm2(c, rhs, &bnorm)) return rc;
    *iters = 0;
    *relres = 0.0;
    if (bnorm == 0.0) return BEM_OK;
    double res = 0.0;
    const int rc = gmres(c, precision, rhs, x, true, tol * bnorm, c->prm.max_iters, iters, &res, true);
    *relres = res / bnorm;
    return rc;
}

extern "C" int bem_solve(bem_ctx* c, int32_t precision, int32_t nrhs, const double* V0,
                         double* u, double tol, int32_t* iters_out, double* relres)
{
    if (!c) return BEM_ERR_ARG;
    if (precision != BEM_FP64 && precision != BEM_MIXED)
        return set_err(c, BEM_ERR_ARG, "precision must be BEM_FP64 or BEM_MIXED");
    if (nrhs < 1 || nrhs > kMaxRhs || !u || !(tol > 0.0))
        return set_err(c, BEM_ERR_ARG, "bem_solve: need 1 <= nrhs <= %d, u != NULL, tol > 0", kMaxRhs);
    if (!V0 && nrhs != 1) return set_err(c, BEM_ERR_ARG, "bem_solve: V0 = NULL needs nrhs = 1");
    const int64_t n = c->nunk;
    const int nreg = (int)c->regions.size();
    cudaStream_t s = c->stream;
    int total_iters = 0;
    int status = BEM_OK;
    for (int r = 0; r < nrhs; ++r) {
        double* x = u + (int64_t)r * n;
        int rc = bem_rhs(c, 1, V0 ? V0 + (int64_t)r * nreg : nullptr, c->bvec);
        if (rc) return rc;
        BEM_CUDA_TRY(c, cudaMemsetAsync(x, 0, n * sizeof(double), s));
        double bnorm;
        if ((rc = norm2(c, c->bvec, &bnorm))) return rc;
        double res = 0.0;
        if (bnorm == 0.0) {
            if (relres) relres[r] = 0.0;
            continue;
        }
        if (precision == BEM_FP64) {
            rc = gmres(c, BEM_FP64, c->bvec, x, true, tol * bnorm, c->prm.max_iters, &total_iters, &res);
            if (rc && rc != BEM_ERR_NOT_CONVERGED) return rc;
            if (rc == BEM_ERR_NOT_CONVERGED) status = rc;
            if (relres) relres[r] = res / bnorm;
            continue;
        }
        // iterative refinement: inner GMRES on the mixed matvec, residual in FP64
        double* d = c->dvec;   // correction of one refinement step
        double* ri = c->ivec;  // outer residual b - A64 x, the inner right-hand side
        BEM_CUDA_TRY(c, cudaMemcpyAsync(ri, c->bvec, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
        double rnorm = bnorm;
        bool converged = false;
        for (int refine = 0; refine < c->prm.max_refine; ++refine) {
            if (rnorm <= tol * bnorm) break;
            // inner accuracy: 1e-5 of the current residual; FP32 far pairs limit it near 1e-7
            const double inner_tol = std::max(1e-5 * rnorm, 0.5 * tol * bnorm);
            BEM_CUDA_TRY(c, cudaMemsetAsync(d, 0, n * sizeof(double), s));
            double ires = 0.0;
            rc = gmres(c, BEM_MIXED, ri, d, true, inner_tol, c->prm.max_iters, &total_iters, &ires);
            if (rc && rc != BEM_ERR_NOT_CONVERGED) return rc;
            k_axpy<<<nb(n), 256, 0, s>>>(x, d, n);
            BEM_LAUNCH_CHECK(c);
            bool upd = false;
            if (c->prm.residual == BEM_RESIDUAL_DF_UPDATE) {
                double dn, xn;
                if ((rc = norm2(c, d, &dn)) || (rc = norm2(c, x, &xn))) return rc;
                upd = dn <= 1e-3 * xn;
            }
            if (upd) {
                // b - A (x + d) = (b - A x) - A d: the correction's mixed product
                if ((rc = apply(c, BEM_MIXED, false, d, c->rvec))) return rc;
                k_sub<<<nb(n), 256, 0, s>>>(ri, c->rvec, n);
                BEM_LAUNCH_CHECK(c);
            } else {
                const int rprec = c->prm.residual == BEM_RESIDUAL_FP64 ? BEM_FP64 : kPrecDF;
                if ((rc = residual(c, rprec, c->bvec, x, ri))) return rc;
            }
            if ((rc = norm2(c, ri, &rnorm))) return rc;
            if (total_iters >= c->prm.max_iters) break;
        }
        if (rnorm <= tol * bnorm) converged = true;
        if (!converged) status = BEM_ERR_NOT_CONVERGED;
        if (relres) relres[r] = rnorm / bnorm;
    }
    if (iters_out) *iters_out = total_iters;
    if (status == BEM_ERR_NOT_CONVERGED)
        return set_err(c, status, "tolerance not reached within the iteration limit");
    return BEM_OK;
}

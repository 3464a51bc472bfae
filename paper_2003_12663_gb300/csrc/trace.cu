// trace.cu -- field lines and the breakdown integral K = int alpha_eff(|E|) ds
// (Sec. 1, Eq. Breakdowncrit): a persistent launch of tracer CTAs, each tracing up
// to kLW lines at a time with the integrator of trace_core.cuh.
#include "trace_core.cuh"

namespace {

using namespace tcore;

// u32 = u rounded to FP32 (the density of the tracer's regular pairs)
__global__ void k_density32(int64_t np, const double* __restrict__ u, float* __restrict__ u32)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < np) u32[i] = __double2float_rn(u[i]);
}

template <bool F32, int Q>
__global__ void __launch_bounds__(kLT)
k_trace(TArgs A, const double* __restrict__ seeds, int64_t L, unsigned long long* __restrict__ next,
        double* __restrict__ K_out, int32_t* __restrict__ st_out, int32_t* __restrict__ ns_out,
        double* __restrict__ xe_out)
{
    __shared__ Round R;
    __shared__ TArgs sA;
    __shared__ int s_int[3];
    run_lines<F32, Q>([&](int) { return A; }, [&](int) { return L; }, 1, L, next, sA, R, s_int,
                      [&](const TArgs& a, Round& r, int, int64_t line) {
                          NoRec rec;
                          double K, xe[3];
                          int st;
                          int64_t ns;
                          trace_line<F32, Q>(a, r, seeds + 3 * line, rec, K, st, ns, xe);
                          if ((threadIdx.x & 31) == 0) {
                              if (K_out) K_out[line] = K;
                              if (st_out) st_out[line] = st;
                              if (ns_out) ns_out[line] = (int32_t)ns;
                              if (xe_out) {
                                  xe_out[3 * line] = xe[0];
                                  xe_out[3 * line + 1] = xe[1];
                                  xe_out[3 * line + 2] = xe[2];
                              }
                          }
                      });
}

template <bool F32>
int launch(bem_ctx* c, const TArgs& A, int64_t L, const double* seeds, double* K, int32_t* st,
           int32_t* ns, double* xe)
{
    BEM_CUDA_TRY(c, cudaMemsetAsync(c->d_line_next, 0, sizeof(unsigned long long), c->stream));
    switch (c->g) {
#define TR_CASE(G, QQ)                                                                           \
    case G: {                                                                                    \
        constexpr size_t fsm = field_smem<F32, QQ>();                                            \
        BEM_CUDA_TRY(c, allow_smem(k_trace<F32, QQ>, fsm));                                      \
        const int ncl = tracer_cluster(c->np, L, c->num_sms, c->prm.trace_cluster);             \
        const unsigned grid = lines_grid(k_trace<F32, QQ>, fsm, c->num_sms, L, ncl);             \
        BEM_CUDA_TRY(c, launch_lines(k_trace<F32, QQ>, grid, fsm, c->stream, ncl, A, seeds, L,   \
                                     c->d_line_next, K, st, ns, xe));                            \
        break;                                                                                   \
    }
        TR_CASE(1, 1) TR_CASE(2, 4) TR_CASE(3, 9) TR_CASE(4, 16) TR_CASE(5, 25) TR_CASE(6, 36)
#undef TR_CASE
        default: return set_err(c, BEM_ERR_ARG, "far_order %d not compiled", c->g);
    }
    BEM_LAUNCH_CHECK(c);
    return BEM_OK;
}

}  // namespace

extern "C" void bem_default_trace_params(bem_trace_params* tp)
{
    if (!tp) return;
    tp->h = 1e-3;
    tp->r_max = 10.0;
    tp->c = 1e-2;
    tp->E0 = 0.5;
    tp->d = 0.1;
    tp->e_floor = 1e-12;
    tp->max_steps = 200000;
}

int trace_args(bem_ctx* c, const bem_trace_params* tp, const double* u, tcore::TArgs* out)
{
    if (c->p1) return set_err(c, BEM_ERR_ARG, "field lines are not built for curved triangles");
    bem_trace_params p;
    if (tp)
        p = *tp;
    else
        bem_default_trace_params(&p);
    if (!(p.h > 0.0) || !(p.r_max > 0.0) || p.max_steps < 0 || !(p.e_floor >= 0.0))
        return set_err(c, BEM_ERR_ARG, "trace parameters: need h > 0, r_max > 0, max_steps >= 0");
    *out = tcore::TArgs{c->np, c->hdr32, c->hdr64, c->node32, c->node64, c->geo, u, c->d_region,
                        c->d_electrode, p.h, p.r_max, p.c, p.E0, p.d, p.e_floor, p.max_steps, c->nrm32,
                        c->u32};
    if (u) {  // the FP32 density of the regular pairs, on the context's stream
        k_density32<<<(unsigned)((c->np + 255) / 256), 256, 0, c->stream>>>(c->np, u, c->u32);
        BEM_LAUNCH_CHECK(c);
    }
    return BEM_OK;
}

extern "C" int bem_trace_lines(bem_ctx* c, int32_t precision, const double* u, int64_t L,
                               const double* seeds, const bem_trace_params* tp, double* K,
                               int32_t* status, int32_t* nsteps, double* xend)
{
    if (!c) return BEM_ERR_ARG;
    if (precision != BEM_FP64 && precision != BEM_MIXED)
        return set_err(c, BEM_ERR_ARG, "precision must be BEM_FP64 or BEM_MIXED");
    if (L < 0 || L > 0x7fffffff || (L > 0 && (!u || !seeds)))
        return set_err(c, BEM_ERR_ARG, "bem_trace_lines: bad L or NULL pointer");
    TArgs A;
    if (int rc = trace_args(c, tp, u, &A)) return rc;
    if (L == 0) return BEM_OK;
    return precision == BEM_MIXED ? launch<true>(c, A, L, seeds, K, status, nsteps, xend)
                                  : launch<false>(c, A, L, seeds, K, status, nsteps, xend);
}

// peak.cu -- measured arithmetic peaks of the GPU the library runs on: the
// denominators of the regular-pair kernels' roofline (FP32 and FP64 fused
// multiply-add rates).  Not part of the paper's method.
//
// Every thread runs kChains independent multiply-add chains (enough to cover the
// pipeline latency at full occupancy) for a given number of iterations; the rate
// is 2 flops per multiply-add lane over the CUDA-event time of the launch.  The
// FP32 form uses Blackwell's paired instruction (fma on float2, two lanes per
// instruction) and the scalar one; the larger rate is the FP32 peak.
#include <algorithm>

#include "bem_internal.cuh"

namespace {

constexpr int kChains = 8;
constexpr int kPeakThreads = 256;

__global__ void __launch_bounds__(kPeakThreads)
k_peak_ffma2(int iters, float a, float b, float* __restrict__ sink)
{
    float2 x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c)
        x[c] = make_float2(threadIdx.x * 1e-7f + c, blockIdx.x * 1e-7f - c);
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
    if (s == 1234.5f) sink[threadIdx.x] = s;  // never true for the arguments used; keeps the chains live
}

__global__ void __launch_bounds__(kPeakThreads)
k_peak_ffma(int iters, float a, float b, float* __restrict__ sink)
{
    float x[2 * kChains];
#pragma unroll
    for (int c = 0; c < 2 * kChains; ++c) x[c] = threadIdx.x * 1e-7f + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k)
#pragma unroll
            for (int c = 0; c < 2 * kChains; ++c) x[c] = __fmaf_rn(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < 2 * kChains; ++c) s += x[c];
    if (s == 1234.5f) sink[threadIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads)
k_peak_dfma(int iters, double a, double b, double* __restrict__ sink)
{
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = threadIdx.x * 1e-7 + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k)
#pragma unroll
            for (int c = 0; c < kChains; ++c) x[c] = __fma_rn(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 1234.5) sink[threadIdx.x] = s;
}

}  // namespace

extern "C" int bem_measure_peaks(double* fp32_tflops, double* fp64_tflops, double* fp32_scalar_tflops)
{
    int dev = 0, sms = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev) != cudaSuccess)
        return set_err(nullptr, BEM_ERR_CUDA, "bem_measure_peaks: no CUDA device");
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    double* sink = nullptr;
    int rc = BEM_OK;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
        cudaMalloc((void**)&sink, kPeakThreads * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        rc = set_err(nullptr, BEM_ERR_CUDA, "bem_measure_peaks: set-up failed");
    }
    // full occupancy: as many resident CTAs per SM as the thread limit allows
    const unsigned blocks = (unsigned)(sms * std::max(1, per_sm / kPeakThreads));
    const double lanes = (double)blocks * kPeakThreads;
    // best of three launches of each kernel, after one warm-up launch
    auto run = [&](int which, int iters) -> double {
        float best = 3e38f;
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, s);
            if (which == 0)
                k_peak_ffma2<<<blocks, kPeakThreads, 0, s>>>(iters, 0.999999f, 1e-7f, (float*)sink);
            else if (which == 1)
                k_peak_ffma<<<blocks, kPeakThreads, 0, s>>>(iters, 0.999999f, 1e-7f, (float*)sink);
            else
                k_peak_dfma<<<blocks, kPeakThreads, 0, s>>>(iters, 0.999999, 1e-7, sink);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) return -1.0;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) best = std::min(best, ms);
        }
        return best;
    };
    if (!rc) {
        // multiply-adds per thread per iteration: 16 x chains (x2 lanes for the paired form)
        const int it32 = 8192, it64 = 256;
        const double t2 = run(0, it32), t1 = run(1, it32), t64 = run(2, it64);
        if (t2 <= 0 || t1 <= 0 || t64 <= 0 || cudaGetLastError() != cudaSuccess) {
            rc = set_err(nullptr, BEM_ERR_CUDA, "bem_measure_peaks: kernel failed");
        } else {
            const double f2 = lanes * it32 * 16.0 * kChains * 2 * 2;       // paired: 2 lanes x 2 flops
            const double f1 = lanes * it32 * 16.0 * (2 * kChains) * 2;
            const double f64 = lanes * it64 * 16.0 * kChains * 2;
            const double r2 = f2 / (t2 * 1e-3) / 1e12, r1 = f1 / (t1 * 1e-3) / 1e12;
            if (fp32_tflops) *fp32_tflops = std::max(r1, r2);
            if (fp32_scalar_tflops) *fp32_scalar_tflops = r1;
            if (fp64_tflops) *fp64_tflops = f64 / (t64 * 1e-3) / 1e12;
        }
    }
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    return rc;
}

// static_field.cu -- bem_eval_field_static: the field at arbitrary points with the
// far-field partial sums kept in a fixed array of the library's static device
// memory instead of memory the call (or its context) provides.
//
// Who this is for: callers that cannot allocate device memory when they need the
// field -- for example a process that hands the rest of the GPU's memory to its own
// arena after start-up, so that any further cudaMalloc fails or is forbidden.  This
// call never allocates, lazily or otherwise.
//
// The scratch array g_field_scratch (8 MiB) is part of the library's device image:
// every GPU that loads the library holds it until the process exits.  Host code
// cannot use the array's name as a device address (in host code it names a host-side
// stand-in), so the device address is looked up once per device with
// cudaGetSymbolAddress, on the first call made with that device current, and then
// passed to the kernels.  The cached address belongs to the device's primary context
// as it was at that first call; a cudaDeviceReset ends that context and leaves the
// address stale (the header says so).
#include <mutex>

#include "bem_internal.cuh"

namespace {

constexpr int64_t kScratchDoubles = (int64_t)1 << 20;  // 8 MiB of far partial sums
constexpr int64_t kMaxPoints = 65536;                  // points per call
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_field_scratch[kScratchDoubles];

std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_field_scratch on the current device (set up once per device).
int scratch_address(bem_ctx* c, double** out)
{
    int dev = -1;
    BEM_CUDA_TRY(c, cudaGetDevice(&dev));
    if (dev != c->device)
        return set_err(c, BEM_ERR_ARG, "bem_eval_field_static: the context's device %d must be current (is %d)",
                       c->device, dev);
    if (dev < 0 || dev >= kMaxDevices)
        return set_err(c, BEM_ERR_ARG, "bem_eval_field_static: device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_field_scratch);
        if (e != cudaSuccess || !p)
            return set_err(c, BEM_ERR_CUDA, "cudaGetSymbolAddress(g_field_scratch) failed: %s",
                           cudaGetErrorString(e));
        g_scratch_ptr[dev] = (double*)p;
    }
    *out = g_scratch_ptr[dev];
    return BEM_OK;
}

}  // namespace

extern "C" int bem_eval_field_static(bem_ctx* c, int32_t precision, const double* u, int64_t M,
                                     const double* pts, double* phi, double* E)
{
    if (!c) return BEM_ERR_ARG;
    if (precision != BEM_FP64 && precision != BEM_MIXED)
        return set_err(c, BEM_ERR_ARG, "precision must be BEM_FP64 or BEM_MIXED");
    if (M < 0 || (M > 0 && (!u || !pts)))
        return set_err(c, BEM_ERR_ARG, "bem_eval_field_static: bad M or NULL pointer");
    if (M > kMaxPoints)
        return set_err(c, BEM_ERR_CAPACITY,
                       "bem_eval_field_static: M = %lld points exceeds the fixed scratch limit of %lld "
                       "points per call", (long long)M, (long long)kMaxPoints);
    if (c->p1) return set_err(c, BEM_ERR_ARG, "bem_eval_field_static: not built for curved triangles");
    double* scratch = nullptr;
    if (int rc = scratch_address(c, &scratch)) return rc;
    if (M == 0) return BEM_OK;
    // the kernels overwrite every partial they later read, so nothing left in the
    // array by an earlier call needs clearing
    int64_t splits = far_splits(c, precision, M);
    splits = std::max<int64_t>(1, std::min<int64_t>(splits, kScratchDoubles / (4 * M)));
    FarTargets T{nullptr, nullptr, nullptr, pts, M};
    int rc = launch_far(c, precision, T, u, 1, 0, (int)splits, scratch);
    if (rc) return rc;
    return launch_points_near(c, precision, M, pts, u, scratch, (int)splits, phi, E);
}

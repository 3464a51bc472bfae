// order.cu -- spatial order of evaluation points.
//
// The packed regular-pair kernel forms target tiles of consecutive points and sums a
// triangle chunk without per-pair classification when the whole tile lies certainly
// outside the chunk's regular-pair sphere (Sec. 4: a pair is regular iff D > eta R).
// Points given in random order make every tile span the whole point cloud, so every
// chunk takes the masked path.  bem_eval_field therefore evaluates each chunk of
// points in a spatial order: the points' bounding box is cut into 16 x 16 x 16 cells,
// the cells are numbered along the Morton (Z-order) curve, and the points are sorted
// by cell with a stable counting sort (equal cells keep their input order).  Every
// step is deterministic: the box is a min/max reduction, the histogram counts are
// order-free, and the scatter ranks points within a cell by input index.  The sums of
// one point do not depend on which other points share its tile except through the
// chunk classification, so the order only decides which tiles run unmasked.
#include <cfloat>

#include "bem_internal.cuh"

namespace {

constexpr int kAxisBits = 4;                       // cells per axis: 16
constexpr int kCells = 1 << (3 * kAxisBits);       // 4096 cells
constexpr int kSortBlock = 1024;                   // points per block of the sort
constexpr int kBoxBlocks = 128;                    // partial boxes
constexpr int kBoxThreads = 256;

// x, y, z cell coordinates (each < 16) interleaved into a 12-bit Morton index
__device__ __forceinline__ int morton3(int x, int y, int z)
{
    int m = 0;
#pragma unroll
    for (int b = 0; b < kAxisBits; ++b)
        m |= (((x >> b) & 1) << (3 * b)) | (((y >> b) & 1) << (3 * b + 1)) | (((z >> b) & 1) << (3 * b + 2));
    return m;
}

// per-block bounding boxes of the points (FP32, rounded like the kernels' targets)
__global__ void k_box_partial(int64_t M, const double* __restrict__ pts, float* __restrict__ part)
{
    __shared__ float s[6][kBoxThreads];
    float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
    for (int64_t i = blockIdx.x * (int64_t)kBoxThreads + threadIdx.x; i < M; i += (int64_t)gridDim.x * kBoxThreads)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float v = __double2float_rn(pts[3 * i + c]);
            lo[c] = fminf(lo[c], v);
            hi[c] = fmaxf(hi[c], v);
        }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        s[c][threadIdx.x] = lo[c];
        s[3 + c][threadIdx.x] = hi[c];
    }
    __syncthreads();
    for (int o = kBoxThreads / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                s[c][threadIdx.x] = fminf(s[c][threadIdx.x], s[c][threadIdx.x + o]);
                s[3 + c][threadIdx.x] = fmaxf(s[3 + c][threadIdx.x], s[3 + c][threadIdx.x + o]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) part[blockIdx.x * 6 + threadIdx.x] = s[threadIdx.x][0];
}

// cell of every point, and the per-block histogram hist[cell * nblk + block]
__global__ void __launch_bounds__(kSortBlock)
k_cells(int64_t M, const double* __restrict__ pts, const float* __restrict__ box_part,
        int32_t* __restrict__ cell, int32_t* __restrict__ hist, int nblk)
{
    __shared__ int s_h[kCells];
    __shared__ float s_box[6];
    if (threadIdx.x < 6) {
        const int c = threadIdx.x;
        float v = box_part[c];
        for (int b = 1; b < kBoxBlocks; ++b)
            v = c < 3 ? fminf(v, box_part[b * 6 + c]) : fmaxf(v, box_part[b * 6 + c]);
        s_box[c] = v;
    }
    for (int k = threadIdx.x; k < kCells; k += kSortBlock) s_h[k] = 0;
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)kSortBlock + threadIdx.x;
    if (i < M) {
        int q[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float ext = s_box[3 + c] - s_box[c];
            const float v = __double2float_rn(pts[3 * i + c]);
            const int k = ext > 0.f ? (int)((v - s_box[c]) * ((float)(1 << kAxisBits) / ext)) : 0;
            q[c] = min(max(k, 0), (1 << kAxisBits) - 1);
        }
        const int m = morton3(q[0], q[1], q[2]);
        cell[i] = m;
        atomicAdd(&s_h[m], 1);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kCells; k += kSortBlock) hist[(int64_t)k * nblk + blockIdx.x] = s_h[k];
}

// exclusive prefix sum of n counts in place (one block: each thread scans a contiguous
// segment, the segment totals are scanned in shared memory)
__global__ void __launch_bounds__(1024) k_scan(int32_t* __restrict__ a, int64_t n)
{
    __shared__ int64_t s[1024];
    const int64_t seg = (n + 1023) / 1024;
    const int64_t b = threadIdx.x * seg, e = min(n, b + seg);
    int64_t sum = 0;
    for (int64_t k = b; k < e; ++k) sum += a[k];
    s[threadIdx.x] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // inclusive Hillis-Steele scan of the totals
        const int64_t v = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
        __syncthreads();
        s[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t run = s[threadIdx.x] - sum;
    for (int64_t k = b; k < e; ++k) {
        const int64_t v = a[k];
        a[k] = (int32_t)run;
        run += v;
    }
}

// stable scatter: the block's points take their cell's next slots in input order,
// warp by warp (within a warp, lanes of the same cell are ranked by lane)
__global__ void __launch_bounds__(kSortBlock)
k_scatter(int64_t M, const double* __restrict__ pts, const int32_t* __restrict__ cell,
          const int32_t* __restrict__ hist, int nblk, double* __restrict__ spts, int32_t* __restrict__ perm)
{
    __shared__ int s_next[kCells + 1];
    for (int k = threadIdx.x; k < kCells; k += kSortBlock) s_next[k] = hist[(int64_t)k * nblk + blockIdx.x];
    if (threadIdx.x == 0) s_next[kCells] = 0;
    const int64_t i = blockIdx.x * (int64_t)kSortBlock + threadIdx.x;
    const int m = i < M ? cell[i] : kCells;  // a lane past the end takes the spare counter
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int w = 0; w < kSortBlock / 32; ++w) {
        __syncthreads();
        if (warp != w) continue;
        const unsigned peers = __match_any_sync(0xffffffffu, m);
        const int pos = s_next[m] + __popc(peers & ((1u << lane) - 1u));
        __syncwarp();
        if (lane == __ffs(peers) - 1) s_next[m] += __popc(peers);
        if (i < M) {
            perm[pos] = (int32_t)i;
            spts[3 * (int64_t)pos] = pts[3 * i];
            spts[3 * (int64_t)pos + 1] = pts[3 * i + 1];
            spts[3 * (int64_t)pos + 2] = pts[3 * i + 2];
        }
    }
}

}  // namespace

int64_t order_hist_len(int64_t max_points)
{
    return (int64_t)kCells * ((max_points + kSortBlock - 1) / kSortBlock);
}

int64_t order_box_len() { return 6 * kBoxBlocks; }

// spts[k] = pts[perm[k]] for k < M, in the cell order above (M <= prm.max_points)
int order_points(bem_ctx* c, int64_t M, const double* pts, double* spts, int32_t* perm)
{
    if (M <= 0) return BEM_OK;
    const int nblk = (int)((M + kSortBlock - 1) / kSortBlock);
    cudaStream_t s = c->stream;
    k_box_partial<<<kBoxBlocks, kBoxThreads, 0, s>>>(M, pts, c->ord_box);
    BEM_LAUNCH_CHECK(c);
    k_cells<<<nblk, kSortBlock, 0, s>>>(M, pts, c->ord_box, c->ord_cell, c->ord_hist, nblk);
    BEM_LAUNCH_CHECK(c);
    k_scan<<<1, 1024, 0, s>>>(c->ord_hist, (int64_t)kCells * nblk);
    BEM_LAUNCH_CHECK(c);
    k_scatter<<<nblk, kSortBlock, 0, s>>>(M, pts, c->ord_cell, c->ord_hist, nblk, spts, perm);
    BEM_LAUNCH_CHECK(c);
    return BEM_OK;
}

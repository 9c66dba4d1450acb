// k_static.cu -- reprojection binning of a caller-held batch without any
// device allocation (afr_reproject_batch_static in include/afr.h).
//
// Some callers cannot call cudaMalloc at the moment they need this step: a
// render thread with a fixed memory budget, a plugin whose host forbids
// allocation in its frame callback, or code issuing work while another
// component owns the allocator. This entry point needs no context: the
// caller passes the batch and the output arrays, and the only scratch (the
// per-pixel counters and the scan's block sums) lives in one file-scope
// device array of fixed size, which every GPU that loads the library holds
// until the process exits.
//
// The scratch address is looked up with cudaGetSymbolAddress once per device,
// on the first call made with that device current, and cached; make that
// first call before any stream capture. The cache is not refreshed after
// cudaDeviceReset (the module may then load at another address), so calls
// made after a device reset are undefined. Every call shares the array and
// leaves its contents behind, so each call clears the counters it uses first;
// calls whose work overlaps on the GPU (other streams, or other host threads)
// race on the array and must be serialised by the caller.
#include <cmath>
#include <mutex>

#include "afr_internal.cuh"

namespace afr {
namespace {

constexpr uint32_t kStaticMaxPixels = 1u << 20;   // width * height up to 1,048,576 (1024 x 1024)
constexpr uint32_t kStaticMaxSamples = 1u << 26;  // batch size up to 67,108,864
constexpr uint32_t kStaticScanTmp = (kStaticMaxPixels + 4095) / 4096 + 2;
constexpr int kMaxDevices = 64;

// [0, kStaticMaxPixels): per-pixel counters, then cursors; the rest: scan block sums
static __device__ __align__(256) uint32_t g_scratch[kStaticMaxPixels + kStaticScanTmp];

std::mutex g_mutex;
uint32_t *g_scratch_ptr[kMaxDevices] = {nullptr};

// Same acceptance rule as afr_insert_samples and same move as afr_reproject.
template <int CT>
__device__ __forceinline__ bool accept_and_move(const float4 *pos, const void *col, const float2 *mo, uint32_t i,
                                                int W, int H, float t_now, float4 &rec, uint32_t &bin) {
    const float4 p = __ldg(pos + i);
    const float3 c = ColorStore<CT>::load(col, i);
    const float2 m = __ldg(mo + i);
    const bool ok = isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(c.x) && isfinite(c.y) &&
                    isfinite(c.z) && isfinite(m.x) && isfinite(m.y) && p.x >= 0.f && p.y >= 0.f && p.x < (float)W &&
                    p.y < (float)H;
    if (!ok) return false;
    const float a = __fsub_rn(t_now, p.z);
    const float xp = __fadd_rn(p.x, __fmul_rn(m.x, a));
    const float yp = __fadd_rn(p.y, __fmul_rn(m.y, a));
    if (!(xp >= 0.f && xp < (float)W && yp >= 0.f && yp < (float)H)) return false;
    const int qx = (int)floorf(xp);
    bin = (uint32_t)(int)floorf(yp) * (uint32_t)W + (uint32_t)qx;
    rec = make_float4(xp, yp, __fmul_rn(a, a), __int_as_float(qx));
    return true;
}

__global__ void k_st_zero(uint32_t *p, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = 0u;
}

template <int CT>
__global__ void __launch_bounds__(256) k_st_count(const float4 *pos, const void *col, const float2 *mo, uint32_t n,
                                                  int W, int H, float t_now, uint32_t *cnt) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float4 rec;
        uint32_t bin;
        if (accept_and_move<CT>(pos, col, mo, i, W, H, t_now, rec, bin)) agg_inc(cnt, bin);
    }
}

// Each moved sample writes its batch index into its bin's list (unordered),
// in seq_out, which the fix-up pass overwrites with the ordered indices.
template <int CT>
__global__ void __launch_bounds__(256) k_st_list(const float4 *pos, const void *col, const float2 *mo, uint32_t n,
                                                 int W, int H, float t_now, const uint32_t *off, uint32_t *cur,
                                                 uint32_t *list) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float4 rec;
        uint32_t bin;
        if (accept_and_move<CT>(pos, col, mo, i, W, H, t_now, rec, bin)) list[off[bin] + agg_inc(cur, bin)] = i;
    }
}

// A sample's rank in its bin is the number of batch indices in the bin's list
// below its own, so the records land in batch order; a bin above
// kSortedBinMax records takes ranks by counting its counter down (arrival
// order). The record's fourth lane holds the batch index until the fix-up.
template <int CT>
__global__ void __launch_bounds__(256) k_st_place(const float4 *pos, const void *col, const float2 *mo, uint32_t n,
                                                  int W, int H, float t_now, const uint32_t *off, uint32_t *cnt,
                                                  const uint32_t *list, float4 *out_rec, void *out_col) {
    using CS = ColorStore<CT>;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float4 rec;
        uint32_t bin;
        if (!accept_and_move<CT>(pos, col, mo, i, W, H, t_now, rec, bin)) continue;
        const uint32_t beg = off[bin], end = off[bin + 1];
        uint32_t rank = 0;
        if (end - beg <= (uint32_t)kSortedBinMax) {
            for (uint32_t k = beg; k < end; ++k) rank += list[k] < i;
        } else {
            rank = atomicSub(cnt + bin, 1u) - 1u;
        }
        rec.w = __uint_as_float(i);
        out_rec[beg + rank] = rec;
        reinterpret_cast<typename CS::T *>(out_col)[beg + rank] = CS::raw(col, i);
    }
}

// Moves each record's batch index to seq_out and puts the bin column back.
__global__ void __launch_bounds__(256) k_st_fix(const uint32_t *off, uint32_t P, float4 *rec, uint32_t *seq) {
    const uint32_t n = off[P];
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        float4 r = rec[e];
        seq[e] = __float_as_uint(r.w);
        r.w = __int_as_float((int)floorf(r.x));
        rec[e] = r;
    }
}

__global__ void k_st_total(const uint32_t *off, uint32_t P, uint32_t *n_frame) { *n_frame = off[P]; }

// Device address of the scratch array for the current device (cached).
AfrStatus scratch_for_current_device(uint32_t **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return AFR_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return AFR_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        uint32_t *ptr = nullptr;
        if (cudaGetSymbolAddress(reinterpret_cast<void **>(&ptr), g_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return AFR_ERR_CUDA;
        }
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return AFR_OK;
}

template <int CT>
cudaError_t run_static(const AfrSampleBatch *b, uint32_t n, int W, int H, float t_now, uint32_t *off, float4 *rec,
                       void *col, uint32_t *seq, uint32_t *n_frame, uint32_t *scratch, cudaStream_t s) {
    const float4 *pos = reinterpret_cast<const float4 *>(b->pos_dev);
    const float2 *mo = reinterpret_cast<const float2 *>(b->motion_dev);
    const void *cin = b->color_dev;
    const uint32_t P = (uint32_t)W * (uint32_t)H;
    uint32_t *cnt = scratch, *scan_tmp = scratch + kStaticMaxPixels;
    const int gp = grid_for(P, 256), gn = grid_for(n, 256);
    k_st_zero<<<gp, 256, 0, s>>>(cnt, P);
    if (n) k_st_count<CT><<<gn, 256, 0, s>>>(pos, cin, mo, n, W, H, t_now, cnt);
    cudaError_t e = scan_exclusive(cnt, off, P, scan_tmp, s);
    if (e != cudaSuccess) return e;
    k_st_zero<<<gp, 256, 0, s>>>(cnt, P);
    if (n) {
        k_st_list<CT><<<gn, 256, 0, s>>>(pos, cin, mo, n, W, H, t_now, off, cnt, seq);
        k_st_place<CT><<<gn, 256, 0, s>>>(pos, cin, mo, n, W, H, t_now, off, cnt, seq, rec, col);
        k_st_fix<<<gn, 256, 0, s>>>(off, P, rec, seq);
    }
    if (n_frame) k_st_total<<<1, 1, 0, s>>>(off, P, n_frame);
    return cudaGetLastError();
}

bool aligned_to(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace
}  // namespace afr

extern "C" AfrStatus afr_reproject_batch_static(const AfrSampleBatch *batch, uint32_t n, int32_t width,
                                                int32_t height, int32_t color_type, float t_now, uint32_t *off_dev,
                                                float *rec_dev, void *col_dev, uint32_t *seq_dev,
                                                uint32_t *n_frame_dev, afr_stream_t stream) {
    using namespace afr;
    if (!batch || !off_dev || !rec_dev || !col_dev || !seq_dev) return AFR_ERR_INVALID_ARG;
    if (width < 1 || height < 1 || color_type < AFR_F32 || color_type > AFR_BF16 || !std::isfinite(t_now))
        return AFR_ERR_INVALID_ARG;
    if ((uint64_t)width * (uint64_t)height > kStaticMaxPixels || n > kStaticMaxSamples) return AFR_ERR_INVALID_ARG;
    const size_t csize = color_type == AFR_F32 ? 16 : 8;
    if (n && (!batch->pos_dev || !batch->color_dev || !batch->motion_dev || !aligned_to(batch->pos_dev, 16) ||
              !aligned_to(batch->color_dev, csize) || !aligned_to(batch->motion_dev, 8)))
        return AFR_ERR_INVALID_ARG;
    if (!aligned_to(rec_dev, 16) || !aligned_to(col_dev, csize)) return AFR_ERR_INVALID_ARG;
    uint32_t *scratch = nullptr;
    AfrStatus st = scratch_for_current_device(&scratch);
    if (st != AFR_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    float4 *rec = reinterpret_cast<float4 *>(rec_dev);
    cudaError_t e;
    switch (color_type) {
        case AFR_F32:
            e = run_static<AFR_F32>(batch, n, width, height, t_now, off_dev, rec, col_dev, seq_dev, n_frame_dev,
                                    scratch, s);
            break;
        case AFR_F16:
            e = run_static<AFR_F16>(batch, n, width, height, t_now, off_dev, rec, col_dev, seq_dev, n_frame_dev,
                                    scratch, s);
            break;
        default:
            e = run_static<AFR_BF16>(batch, n, width, height, t_now, off_dev, rec, col_dev, seq_dev, n_frame_dev,
                                     scratch, s);
            break;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? AFR_ERR_OOM : AFR_ERR_CUDA;
    }
    return AFR_OK;
}

// k_scan.cu -- exclusive prefix sum of uint32 counts (bin offsets of the
// counting sorts in ingest and reprojection). Reduce-then-scan in three
// launches: per-block sums, a single-block scan of those sums, and a
// per-block scan that adds its block's prefix. out has n+1 entries; out[n]
// is the total.
#include "afr_internal.cuh"

namespace afr {
namespace {

constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread; returns the block total
// through *total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *total) {
    __shared__ uint32_t warp_sums[kScanThreads / 32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = warp_incl_scan(v);
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kScanThreads / 32 ? warp_sums[lane] : 0u;
        uint32_t wi = warp_incl_scan(w);
        if (lane < kScanThreads / 32) warp_sums[lane] = wi - w;
        if (lane == kScanThreads / 32 - 1) *total = wi;
    }
    __syncthreads();
    uint32_t r = warp_sums[warp] + incl - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_block_sums(const uint32_t *in, size_t n,
                                                              uint32_t *sums) {
    size_t base = (size_t)blockIdx.x * kScanTile;
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        size_t i = base + (size_t)k * kScanThreads + threadIdx.x;
        if (i < n) acc += in[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ uint32_t ws[kScanThreads / 32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) t += ws[w];
        sums[blockIdx.x] = t;
    }
}

// Scans nb block sums in place (exclusive) with one block; sums[nb] = total.
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(uint32_t *sums, size_t nb) {
    __shared__ uint32_t carry;
    __shared__ uint32_t tot;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (size_t base = 0; base < nb; base += kScanThreads) {
        size_t i = base + threadIdx.x;
        uint32_t v = i < nb ? sums[i] : 0u;
        uint32_t ex = block_excl_scan(v, &tot);
        if (i < nb) sums[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[nb] = carry;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const uint32_t *in, uint32_t *out, size_t n,
                                                              const uint32_t *sums) {
    __shared__ uint32_t tot;
    size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t acc = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        size_t i = base + k;
        v[k] = i < n ? in[i] : 0u;
        acc += v[k];
    }
    uint32_t ex = block_excl_scan(acc, &tot) + sums[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        size_t i = base + k;
        if (i < n) out[i] = ex;
        ex += v[k];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = sums[gridDim.x];
}

}  // namespace

size_t scan_tmp_elems(size_t n) { return (n + kScanTile - 1) / kScanTile + 2; }

cudaError_t scan_exclusive(const uint32_t *in, uint32_t *out, size_t n, uint32_t *tmp, cudaStream_t s) {
    size_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 0) {
        return cudaMemsetAsync(out, 0, sizeof(uint32_t), s);
    }
    k_block_sums<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, tmp);
    k_scan_sums<<<1, kScanThreads, 0, s>>>(tmp, nb);
    k_scan_tiles<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, tmp);
    return cudaGetLastError();
}

}  // namespace afr

// k_feedback.cu -- sections 4, 4.2 and 6.1: finalise the per-tile records
// from the partials of the gradient pass. One block walks all tiles twice:
// the mean number of empty slots over tiles (FP64), then each tile's record
// with its undersampling measure u = 1 - min(1, m * mean_empty / empty).
#include "afr_internal.cuh"

namespace afr {
namespace {

constexpr int kFbThreads = 1024;

__global__ void __launch_bounds__(kFbThreads) k_finalize(int W, int H, int S, int ntx, int ntiles, int b, float m,
                                                         const TilePartial *__restrict__ tiles,
                                                         AfrTileStats *__restrict__ out) {
    __shared__ double sh[kFbThreads / 32];
    __shared__ double mean_empty;
    double acc = 0.0;
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        int tx = t % ntx, ty = t / ntx;
        double A = (double)(min(S, W - tx * S) * min(S, H - ty * S));
        acc += A * b - tiles[t].n;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        mean_empty = s / ntiles;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        int tx = t % ntx, ty = t / ntx;
        double A = (double)(min(S, W - tx * S) * min(S, H - ty * S));
        TilePartial tp = tiles[t];
        double empty = A * b - tp.n;
        AfrTileStats o;
        o.n = (uint32_t)tp.n;
        o.empty_slots = (uint32_t)empty;
        o.mean_L = tp.sw > 0.0 ? (float)tp.mean : 0.f;
        o.var_L = tp.sw > 0.0 ? (float)(tp.m2 / tp.sw) : 0.f;
        o.mean_Gx = tp.nonempty > 0.0 ? (float)(tp.sgx / tp.nonempty) : 0.f;
        o.mean_Gy = tp.nonempty > 0.0 ? (float)(tp.sgy / tp.nonempty) : 0.f;
        o.mean_Gt = tp.nonempty > 0.0 ? (float)(tp.sgt / tp.nonempty) : 0.f;
        double r = empty > 0.0 ? (double)m * mean_empty / empty : 0.0;
        o.u = empty > 0.0 ? (float)(1.0 - (r < 1.0 ? r : 1.0)) : 0.f;
        out[t] = o;
    }
}

}  // namespace

cudaError_t launch_feedback(AfrContext *c, AfrTileStats *out, cudaStream_t s) {
    k_finalize<<<1, kFbThreads, 0, s>>>(c->W, c->H, c->S, c->ntx, c->ntiles, c->b, c->cfg.undersample_m, c->tiles,
                                        out);
    return cudaGetLastError();
}

}  // namespace afr

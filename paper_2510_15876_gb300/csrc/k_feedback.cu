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

// Sum of sample ages max(0, t_now - t) over each tile's resident samples
// (the queue's count newest slots of every pixel), one block per tile.
__global__ void __launch_bounds__(256) k_tile_age(int W, int H, int S, int ntx, int b, float t_now,
                                                  const uint32_t *__restrict__ state, const float *__restrict__ r_t,
                                                  double *__restrict__ age_sum) {
    __shared__ double sh[8];
    const int tile = blockIdx.x;
    const int x0 = (tile % ntx) * S, y0 = (tile / ntx) * S;
    const int tw = min(S, W - x0), th = min(S, H - y0);
    double acc = 0.0;
    for (int k = threadIdx.x; k < tw * th; k += blockDim.x) {
        const size_t p = (size_t)(y0 + k / tw) * W + x0 + k % tw;
        const uint32_t st = state[p];
        const int cnt = (int)(st & 0xFFFFu), head = (int)(st >> 16);
        for (int j = 0; j < cnt; ++j) {
            const int sl = ((head - 1 - j) % b + b) % b;
            const double a = (double)t_now - (double)__ldg(r_t + p * b + sl);
            acc += a > 0.0 ? a : 0.0;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        age_sum[tile] = t;
    }
}

template <int N>
__device__ __forceinline__ void block_sum(double (&v)[N], double (*sh)[kFbThreads / 32]) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
        double x = v[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0) sh[i][threadIdx.x >> 5] = x;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N; ++i) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[i][w];
        v[i] = t;
    }
    __syncthreads();
}

// Sections 6.1 and 4.1: tile error shares and gain control, one block.
__global__ void __launch_bounds__(kFbThreads) k_tile_error(int W, int H, int S, int ntx, int ntiles, int b, float m,
                                                           double kappa, double lambda, double importance, double eps,
                                                           const TilePartial *__restrict__ tiles,
                                                           const double *__restrict__ age_sum,
                                                           const uint32_t *__restrict__ occluded,
                                                           float *__restrict__ E, AfrGain *__restrict__ gain) {
    __shared__ double sh[8][kFbThreads / 32];
    auto area = [&](int t) {
        const int tx = t % ntx, ty = t / ntx;
        return (double)(min(S, W - tx * S) * min(S, H - ty * S));
    };
    double e1[1] = {0.0};
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) e1[0] += area(t) * b - tiles[t].n;
    block_sum(e1, sh);
    const double mean_empty = e1[0] / ntiles;
    auto var_u_o = [&](int t, double &v, double &u, double &o) {
        const TilePartial tp = tiles[t];
        const double A = area(t), empty = A * b - tp.n;
        v = tp.sw > 0.0 ? tp.m2 / tp.sw : 0.0;
        const double r = empty > 0.0 ? (double)m * mean_empty / empty : 0.0;
        u = empty > 0.0 ? 1.0 - (r < 1.0 ? r : 1.0) : 0.0;
        o = occluded ? (double)occluded[t] / (A * b) : 0.0;
    };
    // sums: v, u, o, spatial gradient, temporal gradient, non-empty pixels, tile mean ages, tiles with samples
    double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        double v, u, o;
        var_u_o(t, v, u, o);
        const TilePartial tp = tiles[t];
        acc[0] += v;
        acc[1] += u;
        acc[2] += o;
        acc[3] += 0.5 * (tp.sgx + tp.sgy);
        acc[4] += tp.sgt;
        acc[5] += tp.nonempty;
        if (tp.n > 0.0) {
            acc[6] += age_sum[t] / tp.n;
            acc[7] += 1.0;
        }
    }
    block_sum(acc, sh);
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        double v, u, o;
        var_u_o(t, v, u, o);
        double e = 0.0;
        if (acc[0] > 0.0) e += kappa * v / acc[0];
        if (acc[1] > 0.0) e += lambda * u / acc[1];
        if (occluded && acc[2] > 0.0) e += (1.0 - kappa - lambda) * o / acc[2];
        E[t] = (float)(area(t) * e);
    }
    if (threadIdx.x == 0 && gain) {
        const double dcds = acc[5] > 0.0 ? acc[3] / acc[5] : 0.0, dcdt = acc[5] > 0.0 ? acc[4] / acc[5] : 0.0;
        const double T = acc[7] > 0.0 ? acc[6] / acc[7] : 0.0;
        const double Sw = importance * dcdt * T / (dcds > eps ? dcds : eps);
        const double P = (double)W * H;
        double N = Sw > 0.0 ? P / (Sw * Sw) : P;
        N = N < 1.0 ? 1.0 : (N > P ? P : N);
        AfrGain g;
        g.dC_ds = (float)dcds;
        g.dC_dt = (float)dcdt;
        g.mean_age = (float)T;
        g.tile_width = (float)Sw;
        g.tile_count = (float)N;
        *gain = g;
    }
}

}  // namespace

cudaError_t launch_tile_error(AfrContext *c, float kappa, float lambda, float importance, const uint32_t *occluded,
                              float *E, AfrGain *gain, cudaStream_t s) {
    k_tile_age<<<c->ntiles, 256, 0, s>>>(c->W, c->H, c->S, c->ntx, c->b, c->grads_t, c->r_state, c->r_t,
                                         c->tile_age);
    k_tile_error<<<1, kFbThreads, 0, s>>>(c->W, c->H, c->S, c->ntx, c->ntiles, c->b, c->cfg.undersample_m, kappa,
                                          lambda, importance, c->cfg.eps_grad, c->tiles, c->tile_age, occluded, E,
                                          gain);
    return cudaGetLastError();
}

cudaError_t launch_feedback(AfrContext *c, AfrTileStats *out, cudaStream_t s) {
    k_finalize<<<1, kFbThreads, 0, s>>>(c->W, c->H, c->S, c->ntx, c->ntiles, c->b, c->cfg.undersample_m, c->tiles,
                                        out);
    return cudaGetLastError();
}

}  // namespace afr

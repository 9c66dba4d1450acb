// k_feedback.cu -- sections 4, 4.2 and 6.1: finalise the per-tile records
// from the partials of the gradient pass (the mean number of empty slots over
// tiles, then each tile's record with its undersampling measure
// u = 1 - min(1, m * mean_empty / empty)), and the tile error E with the gain
// control of section 4.1. Counts are summed as integers and the rest runs in
// FP32: FP64 issues at 1/64 of the FP32 rate on this part, and every output
// is FP32.
#include "afr_internal.cuh"

namespace afr {
namespace {

constexpr int kFbThreads = 1024;
constexpr int kFinThreads = 256;

__device__ __forceinline__ uint32_t tile_area(int t, int W, int H, int S, int ntx) {
    const int tx = t % ntx, ty = t / ntx;
    return (uint32_t)(min(S, W - tx * S) * min(S, H - ty * S));
}

// Every block sums the empty slots of all tiles (an exact integer sum, the
// same in every block), then writes the records of its own kFinThreads tiles.
__global__ void __launch_bounds__(kFinThreads) k_finalize(int W, int H, int S, int ntx, int ntiles, int b, float m,
                                                          const TilePartial *__restrict__ tiles,
                                                          AfrTileStats *__restrict__ out) {
    __shared__ unsigned long long sh[kFinThreads / 32];
    __shared__ float mean_empty;
    unsigned long long acc = 0ull;
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x)
        acc += (unsigned long long)tile_area(t, W, H, S, ntx) * (uint32_t)b - tiles[t].n;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long s = 0ull;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        mean_empty = (float)s / (float)ntiles;
    }
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < ntiles) {
        const TilePartial tp = tiles[t];
        const uint32_t empty = tile_area(t, W, H, S, ntx) * (uint32_t)b - tp.n;
        const float sw = (float)tp.sw, ne = (float)tp.nonempty;
        AfrTileStats o;
        o.n = tp.n;
        o.empty_slots = empty;
        o.mean_L = sw > 0.f ? (float)tp.mean : 0.f;
        o.var_L = sw > 0.f ? (float)tp.m2 / sw : 0.f;
        o.mean_Gx = tp.nonempty ? tp.sgx / ne : 0.f;
        o.mean_Gy = tp.nonempty ? tp.sgy / ne : 0.f;
        o.mean_Gt = tp.nonempty ? tp.sgt / ne : 0.f;
        const float r = empty ? m * mean_empty / (float)empty : 0.f;
        o.u = empty ? 1.f - fminf(r, 1.f) : 0.f;
        out[t] = o;
    }
}

// Per-tile terms of the tile error, one block per tile: the sum of sample
// ages max(0, t_now - t) over the tile's resident samples (the queue's count
// newest slots of every pixel), then, by one thread, the tile's terms that do
// not depend on other tiles. A tile row's slots are contiguous (tw pixels x b
// slots): each thread keeps its slot columns and walks the rows, loading a
// slot's time beside its pixel's queue state (a warp reads 128 contiguous
// bytes of times) so that the loads of successive rows overlap. Ages are
// summed in FP32 over at most 32 rows of one slot column (32 ages, each at
// most the window); those sums are added as double-float values (TwoSum
// additions), per thread and by a tree over the block.
struct alignas(16) TileTerm {
    float v;           // luminance variance
    float o;           // occluded share of the tile's slots
    float inv_empty;   // 1 / empty slots (0 without empty slots)
    float age;         // mean sample age (unused without samples)
    float sg, sgt;     // spatial and temporal gradient sums over non-empty pixels
    uint32_t empty, nonempty, has_samples, pad[3];
};
static_assert(sizeof(TileTerm) <= 64, "fits the 64 bytes a tile the context holds");

__global__ void __launch_bounds__(256) k_tile_terms(int W, int H, int S, int ntx, int b, float t_now,
                                                    const uint32_t *__restrict__ state, const float *__restrict__ r_t,
                                                    const TilePartial *__restrict__ tiles,
                                                    const uint32_t *__restrict__ occluded,
                                                    TileTerm *__restrict__ terms) {
    __shared__ float2 sh[8];
    const int tile = blockIdx.x;
    const int x0 = (tile % ntx) * S, y0 = (tile / ntx) * S;
    const int tw = min(S, W - x0), th = min(S, H - y0);
    const int row_slots = tw * b;
    dfloat d{0.f, 0.f};   // double-float: each chunk's FP32 sum added exactly (TwoSum)
    for (int k = threadIdx.x; k < row_slots; k += blockDim.x) {
        const int px = k / b, sl = k - px * b;
        const size_t p0 = (size_t)y0 * W + x0 + px;
        for (int r0 = 0; r0 < th; r0 += 32) {
            const int r1 = min(th, r0 + 32);
            float acc = 0.f;
#pragma unroll 8
            for (int r = r0; r < r1; ++r) {
                const size_t p = p0 + (size_t)r * W;
                const uint32_t st = __ldg(state + p);
                const float t = __ldg(r_t + p * b + sl);
                int age_rank = (int)(st >> 16) - 1 - sl;
                if (age_rank < 0) age_rank += b;
                const float a = t_now - t;
                acc += (age_rank < (int)(st & 0xFFFFu) && a > 0.f) ? a : 0.f;
            }
            d = df_add(d, dfloat{acc, 0.f});
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        d = df_add(d, dfloat{__shfl_xor_sync(0xffffffffu, d.h, o), __shfl_xor_sync(0xffffffffu, d.l, o)});
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = make_float2(d.h, d.l);
    __syncthreads();
    if (threadIdx.x < 32) {
        const float2 v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : make_float2(0.f, 0.f);
        dfloat xd{v.x, v.y};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            xd = df_add(xd, dfloat{__shfl_xor_sync(0xffffffffu, xd.h, o), __shfl_xor_sync(0xffffffffu, xd.l, o)});
        const float x = __fadd_rn(xd.h, xd.l);
        if (threadIdx.x == 0) {
            const TilePartial tp = tiles[tile];
            const uint32_t slots = (uint32_t)(tw * th) * (uint32_t)b, empty = slots - tp.n;
            const float sw = (float)tp.sw;
            TileTerm tt;
            tt.v = sw > 0.f ? (float)tp.m2 / sw : 0.f;
            tt.o = occluded ? (float)occluded[tile] / (float)slots : 0.f;
            tt.inv_empty = empty ? 1.f / (float)empty : 0.f;
            tt.age = tp.n ? x / (float)tp.n : 0.f;
            tt.sg = 0.5f * (tp.sgx + tp.sgy);
            tt.sgt = tp.sgt;
            tt.empty = empty;
            tt.nonempty = tp.nonempty;
            tt.has_samples = tp.n ? 1u : 0u;
            tt.pad[0] = tt.pad[1] = tt.pad[2] = 0u;
            terms[tile] = tt;
        }
    }
}

// Sum of each of N values over the block's kFbThreads threads: warp sums by
// shuffles, then warp 0 sums the warps' partials and shares the totals.
template <typename T, int N>
__device__ __forceinline__ void block_sum(T (&v)[N], T (*sh)[kFbThreads / 32]) {
    static_assert(kFbThreads == 1024, "warp 0 sums one partial per lane");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < N; ++i) {
        T x = v[i];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) sh[i][warp] = x;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            T x = sh[i][lane];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == 0) sh[i][0] = x;
        }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = sh[i][0];
    __syncthreads();
}

// Sections 6.1 and 4.1: tile error shares and gain control, one block over
// the per-tile terms. The counts (empty slots, non-empty pixels, tiles with
// samples) are summed as integers, exactly; the rest are tree sums in FP32.
__global__ void __launch_bounds__(kFbThreads) k_tile_error(int W, int H, int S, int ntx, int ntiles, float m,
                                                           float kappa, float lambda, float importance, float eps,
                                                           const TileTerm *__restrict__ terms, bool has_occlusion,
                                                           float *__restrict__ E, AfrGain *__restrict__ gain) {
    __shared__ unsigned long long shi[3][kFbThreads / 32];
    __shared__ float sh[6][kFbThreads / 32];
    __shared__ float scal[4];   // m mean_empty, then the weights of v, u, o (one thread divides)
    unsigned long long cnt[3] = {0ull, 0ull, 0ull};   // empty slots, non-empty pixels, tiles with samples
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        cnt[0] += terms[t].empty;
        cnt[1] += terms[t].nonempty;
        cnt[2] += terms[t].has_samples;
    }
    block_sum(cnt, shi);
    if (threadIdx.x == 0) scal[0] = m * ((float)cnt[0] / (float)ntiles);
    __syncthreads();
    const float m_mean_empty = scal[0];
    // u = 1 - min(1, m mean_empty / empty), 0 without empty slots
    auto undersampling = [&](const TileTerm &tt) {
        return tt.empty ? 1.f - fminf(m_mean_empty * tt.inv_empty, 1.f) : 0.f;
    };
    // sums: v, u, o, spatial gradient, temporal gradient, tile mean ages
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        const TileTerm tt = terms[t];
        acc[0] += tt.v;
        acc[1] += undersampling(tt);
        acc[2] += tt.o;
        acc[3] += tt.sg;
        acc[4] += tt.sgt;
        acc[5] += tt.has_samples ? tt.age : 0.f;
    }
    block_sum(acc, sh);
    // E = s (kappa v / sum v + lambda u / sum u + (1 - kappa - lambda) o / sum o)
    if (threadIdx.x == 0) {
        scal[1] = acc[0] > 0.f ? kappa / acc[0] : 0.f;
        scal[2] = acc[1] > 0.f ? lambda / acc[1] : 0.f;
        scal[3] = has_occlusion && acc[2] > 0.f ? (1.f - kappa - lambda) / acc[2] : 0.f;
    }
    __syncthreads();
    const float wv = scal[1], wu = scal[2], wo = scal[3];
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        const TileTerm tt = terms[t];
        const int tx = t % ntx, ty = t / ntx;
        const float A = (float)(min(S, W - tx * S) * min(S, H - ty * S));
        E[t] = A * (wv * tt.v + wu * undersampling(tt) + wo * tt.o);
    }
    if (threadIdx.x == 0 && gain) {
        const float nonempty = (float)cnt[1];
        const float dcds = cnt[1] ? acc[3] / nonempty : 0.f, dcdt = cnt[1] ? acc[4] / nonempty : 0.f;
        const float T = cnt[2] ? acc[5] / (float)cnt[2] : 0.f;
        const float Sw = importance * dcdt * T / (dcds > eps ? dcds : eps);
        const float P = (float)W * (float)H;
        float N = Sw > 0.f ? P / (Sw * Sw) : P;
        N = N < 1.f ? 1.f : (N > P ? P : N);
        AfrGain g;
        g.dC_ds = dcds;
        g.dC_dt = dcdt;
        g.mean_age = T;
        g.tile_width = Sw;
        g.tile_count = N;
        *gain = g;
    }
}

}  // namespace

cudaError_t launch_tile_error(AfrContext *c, float kappa, float lambda, float importance, const uint32_t *occluded,
                              float *E, AfrGain *gain, cudaStream_t s) {
    TileTerm *terms = reinterpret_cast<TileTerm *>(c->tile_terms);
    k_tile_terms<<<c->ntiles, 256, 0, s>>>(c->W, c->H, c->S, c->ntx, c->b, c->grads_t, c->r_state, c->r_t, c->tiles,
                                           occluded, terms);
    k_tile_error<<<1, kFbThreads, 0, s>>>(c->W, c->H, c->S, c->ntx, c->ntiles, c->cfg.undersample_m, kappa, lambda,
                                          importance, c->cfg.eps_grad, terms, occluded != nullptr, E, gain);
    return cudaGetLastError();
}

cudaError_t launch_feedback(AfrContext *c, AfrTileStats *out, cudaStream_t s) {
    k_finalize<<<(c->ntiles + kFinThreads - 1) / kFinThreads, kFinThreads, 0, s>>>(
        c->W, c->H, c->S, c->ntx, c->ntiles, c->b, c->cfg.undersample_m, c->tiles, out);
    return cudaGetLastError();
}

}  // namespace afr

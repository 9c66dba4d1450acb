// k_gradients.cu -- sections 4 and 4.1 on the deep buffer.
//
//  pixel pass   (thread per pixel): reads the pixel's queue newest first,
//               age weights exp(-3.47 a), weighted mean luminance and its
//               weighted spread (per-pixel moments for the tile variance),
//               and the temporal gradient over the queue sorted by time.
//  spatial pass (thread per pixel): G_x, G_y from the four neighbours' means.
//  tile pass    (block per tile): merges per-pixel moments (FP32, or FP64
//               once the tile holds more than 4096 samples) and sums the
//               gradients for the tile record.
#include "afr_internal.cuh"

namespace afr {
namespace {

template <int CT, int B>
__global__ void __launch_bounds__(128) k_pixel(int P, int b, float t_now, const uint32_t *__restrict__ state,
                                               const float *__restrict__ r_t, const uint32_t *__restrict__ r_seq,
                                               const void *__restrict__ r_col, float *__restrict__ lbar,
                                               float4 *__restrict__ pstat) {
    using CS = ColorStore<CT>;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        uint32_t st = __ldg(state + p);
        int n = (int)(st & 0xFFFFu), h = (int)(st >> 16);
        if (n == 0) {
            lbar[p] = __int_as_float(0x7fc00000);
            pstat[p] = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        float T[B], L[B], Wt[B];
        uint32_t Q[B];
        float sw = 0.f, swl = 0.f;
#pragma unroll
        for (int k = 0; k < B; ++k) {
            if (k < n) {
                int s = h - 1 - k;
                if (s < 0) s += b;
                size_t i = (size_t)p * b + s;
                T[k] = __ldg(r_t + i);
                Q[k] = __ldg(r_seq + i);
                L[k] = luminance(CS::load(r_col, i));
                float a = fmaxf(t_now - T[k], 0.f);
                Wt[k] = expf(-kAgeDecay * a);
                sw += Wt[k];
                swl = fmaf(Wt[k], L[k], swl);
            } else {
                T[k] = -INFINITY;
                Q[k] = 0u;
                L[k] = 0.f;
                Wt[k] = 0.f;
            }
        }
        float mean = swl / sw;
        float m2 = 0.f;
#pragma unroll
        for (int k = 0; k < B; ++k) {
            float d = L[k] - mean;
            m2 = fmaf(Wt[k] * d, d, m2);
        }
        // newest first by time, equal times newest first by sequence number;
        // queues filled in time order are already sorted
        bool sorted = true;
#pragma unroll
        for (int k = 0; k + 1 < B; ++k)
            if (k + 1 < n) sorted &= (T[k] > T[k + 1]) || (T[k] == T[k + 1] && Q[k] > Q[k + 1]);
        if (!sorted) {
#pragma unroll
            for (int r = 0; r < B; ++r) {
#pragma unroll
                for (int k = (r & 1); k + 1 < B; k += 2) {
                    bool sw_ = (T[k] < T[k + 1]) || (T[k] == T[k + 1] && Q[k] < Q[k + 1]);
                    if (sw_) {
                        float tt = T[k]; T[k] = T[k + 1]; T[k + 1] = tt;
                        uint32_t qq = Q[k]; Q[k] = Q[k + 1]; Q[k + 1] = qq;
                        float ll = L[k]; L[k] = L[k + 1]; L[k + 1] = ll;
                        float ww = Wt[k]; Wt[k] = Wt[k + 1]; Wt[k + 1] = ww;
                    }
                }
            }
        }
        float num = 0.f, den = 0.f;
#pragma unroll
        for (int k = 0; k + 1 < B; ++k) {
            if (k + 1 < n) {
                num = fmaf(Wt[k], fabsf(L[k] - L[k + 1]), num);
                den = fmaf(Wt[k], T[k] - T[k + 1], den);
            }
        }
        float gt = (n >= 2 && den > 0.f) ? num / den : 0.f;
        lbar[p] = mean;
        pstat[p] = make_float4(sw, mean, m2, gt);
    }
}

__global__ void __launch_bounds__(256) k_spatial(int W, int H, const float *__restrict__ lbar,
                                                 const float4 *__restrict__ pstat, float4 *__restrict__ grad) {
    int P = W * H;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        int x = p % W, y = p / W;
        float l = __ldg(lbar + p);
        float gt = __ldg(&pstat[p].w);
        if (isnan(l)) {
            grad[p] = make_float4(0.f, 0.f, 0.f, l);
            continue;
        }
        float sx = 0.f, sy = 0.f;
        int mx = 0, my = 0;
        float v;
        if (x > 0 && !isnan(v = __ldg(lbar + p - 1))) { sx += fabsf(l - v); ++mx; }
        if (x + 1 < W && !isnan(v = __ldg(lbar + p + 1))) { sx += fabsf(l - v); ++mx; }
        if (y > 0 && !isnan(v = __ldg(lbar + p - W))) { sy += fabsf(l - v); ++my; }
        if (y + 1 < H && !isnan(v = __ldg(lbar + p + W))) { sy += fabsf(l - v); ++my; }
        grad[p] = make_float4(mx ? sx / mx : 0.f, my ? sy / my : 0.f, gt, l);
    }
}

template <typename R>
struct Moments {
    R w, mean, m2;
    __device__ __forceinline__ void merge(R w2, R mean2, R m22) {
        R wt = w + w2;
        if (wt > R(0)) {
            R d = mean2 - mean;
            mean = mean + d * (w2 / wt);
            m2 = m2 + m22 + d * d * (w * w2 / wt);
            w = wt;
        }
    }
};

template <typename R>
__device__ Moments<R> block_merge(Moments<R> m) {
    // warp tree merge then across warps through shared memory
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        R w2 = __shfl_xor_sync(0xffffffffu, m.w, o);
        R mu2 = __shfl_xor_sync(0xffffffffu, m.mean, o);
        R s2 = __shfl_xor_sync(0xffffffffu, m.m2, o);
        m.merge(w2, mu2, s2);
    }
    __shared__ R sh[3][8];
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sh[0][warp] = m.w; sh[1][warp] = m.mean; sh[2][warp] = m.m2; }
    __syncthreads();
    Moments<R> r{R(0), R(0), R(0)};
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r.merge(sh[0][k], sh[1][k], sh[2][k]);
    __syncthreads();
    return r;
}

__device__ __forceinline__ float block_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __shared__ float sh[8];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    float r = 0.f;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
    __syncthreads();
    return r;
}

__device__ __forceinline__ uint32_t block_sum_u(uint32_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __shared__ uint32_t sh[8];
    __shared__ uint32_t tot;
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t r = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) r += sh[k];
        tot = r;
    }
    __syncthreads();
    return tot;
}

template <typename R>
__device__ __forceinline__ Moments<R> tile_moments(int A, int tw, int W, int x0, int y0,
                                                   const uint32_t *__restrict__ state,
                                                   const float4 *__restrict__ pstat) {
    Moments<R> m{R(0), R(0), R(0)};
    for (int k = threadIdx.x; k < A; k += blockDim.x) {
        int p = (y0 + k / tw) * W + x0 + k % tw;
        if ((__ldg(state + p) & 0xFFFFu) == 0) continue;
        float4 ps = __ldg(pstat + p);
        m.merge((R)ps.x, (R)ps.y, (R)ps.z);
    }
    return block_merge(m);
}

__global__ void __launch_bounds__(256) k_tiles(int W, int H, int S, int ntx, const uint32_t *__restrict__ state,
                                               const float4 *__restrict__ pstat, const float4 *__restrict__ grad,
                                               TilePartial *__restrict__ tiles) {
    int tile = blockIdx.x;
    int tx = tile % ntx, ty = tile / ntx;
    int x0 = tx * S, y0 = ty * S;
    int tw = min(S, W - x0), th = min(S, H - y0);
    int A = tw * th;
    uint32_t n = 0, ne = 0;
    float gx = 0.f, gy = 0.f, gtt = 0.f;
    for (int k = threadIdx.x; k < A; k += blockDim.x) {
        int p = (y0 + k / tw) * W + x0 + k % tw;
        uint32_t c = __ldg(state + p) & 0xFFFFu;
        if (c == 0) continue;
        n += c;
        ++ne;
        float4 g = __ldg(grad + p);
        gx += g.x;
        gy += g.y;
        gtt += g.z;
    }
    uint32_t ntot = block_sum_u(n);
    TilePartial out;
    if (ntot > (uint32_t)kSortedBinMax) {   // more than 4096 samples: FP64 merge
        Moments<double> r = tile_moments<double>(A, tw, W, x0, y0, state, pstat);
        out.sw = r.w; out.mean = r.mean; out.m2 = r.m2;
    } else {
        Moments<float> r = tile_moments<float>(A, tw, W, x0, y0, state, pstat);
        out.sw = r.w; out.mean = r.mean; out.m2 = r.m2;
    }
    float sgx = block_sum_f(gx), sgy = block_sum_f(gy), sgt = block_sum_f(gtt);
    uint32_t nne = block_sum_u(ne);
    if (threadIdx.x == 0) {
        out.n = (double)ntot;
        out.nonempty = (double)nne;
        out.sgx = sgx;
        out.sgy = sgy;
        out.sgt = sgt;
        tiles[tile] = out;
    }
}

template <int CT>
cudaError_t launch_pixel(AfrContext *c, float t_now, cudaStream_t s) {
    int g = grid_for(c->P, 128, 152 * 64);
    if (c->b <= 4)
        k_pixel<CT, 4><<<g, 128, 0, s>>>(c->P, c->b, t_now, c->r_state, c->r_t, c->r_seq, c->r_col, c->lbar, c->pstat);
    else if (c->b <= 8)
        k_pixel<CT, 8><<<g, 128, 0, s>>>(c->P, c->b, t_now, c->r_state, c->r_t, c->r_seq, c->r_col, c->lbar, c->pstat);
    else if (c->b <= 16)
        k_pixel<CT, 16><<<g, 128, 0, s>>>(c->P, c->b, t_now, c->r_state, c->r_t, c->r_seq, c->r_col, c->lbar, c->pstat);
    else
        k_pixel<CT, 32><<<g, 128, 0, s>>>(c->P, c->b, t_now, c->r_state, c->r_t, c->r_seq, c->r_col, c->lbar, c->pstat);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_gradients(AfrContext *c, float t_now, cudaStream_t s) {
    cudaError_t e;
    switch (c->ct) {
        case AFR_F32: e = launch_pixel<AFR_F32>(c, t_now, s); break;
        case AFR_F16: e = launch_pixel<AFR_F16>(c, t_now, s); break;
        default: e = launch_pixel<AFR_BF16>(c, t_now, s); break;
    }
    if (e != cudaSuccess) return e;
    k_spatial<<<grid_for(c->P, 256), 256, 0, s>>>(c->W, c->H, c->lbar, c->pstat, c->grad);
    k_tiles<<<c->ntiles, 256, 0, s>>>(c->W, c->H, c->S, c->ntx, c->r_state, c->pstat, c->grad, c->tiles);
    return cudaGetLastError();
}

}  // namespace afr

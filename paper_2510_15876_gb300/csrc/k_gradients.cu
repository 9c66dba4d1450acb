// k_gradients.cu -- sections 4 and 4.1 on the deep buffer.
//
//  pixel pass   (a group of lanes per pixel, several queue slots each): age
//               weights exp(-3.47 a), weighted mean luminance and its weighted
//               spread (per-pixel moments for the tile variance), and the
//               temporal gradient over the queue sorted by time.
//  tile pass    (block per tile): G_x, G_y from the four neighbours' means,
//               the gradient sums and the merged per-pixel moments (FP32, or
//               FP64 once the tile holds more than 4096 samples).
#include "afr_internal.cuh"

namespace afr {
namespace {

// Group of L = G / S lanes per pixel (G = queue depth rounded up to a power
// of two), S queue entries per lane: entry k (0 the newest) sits in lane
// k mod L, register k / L, so the loads of a warp stay contiguous per pixel and
// a warp serves 32 S / G pixels; sums, the time sort and the pairwise
// differences use shuffles within the group.
template <int L>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, L);
    return v;
}

// The value of entry k + 1 for each of a lane's entries k = r L + l.
template <int L, int S, typename V>
__device__ __forceinline__ void next_entry(const V (&v)[S], V (&nv)[S], int l) {
#pragma unroll
    for (int r = 0; r < S; ++r) {
        const V d = __shfl_down_sync(0xffffffffu, v[r], 1, L);
        if (r + 1 < S) {
            const V w = __shfl_sync(0xffffffffu, v[r + 1], 0, L);   // entry (r + 1) L follows entry r L + L - 1
            nv[r] = l == L - 1 ? w : d;
        } else {
            nv[r] = d;
        }
    }
}

struct Entry {
    float T, w, cx, cy, cz;
    uint32_t Q;
};

__device__ __forceinline__ bool newer(const Entry &a, const Entry &b) {   // descending order by (T, Q)
    return (a.T > b.T) || (a.T == b.T && a.Q > b.Q);
}

// Luminance differences carry the gradients: the spatial gradient is a
// difference of neighbouring pixel means and the temporal one a difference
// of consecutive luminances, both far smaller than the luminances. So each
// pixel takes the luminance of its newest sample, in double-float, as its
// reference L_r, and every sample its deviation d = L - L_r in FP32 from the
// colour differences (exact when the colours are within a factor 2, else
// rounded once), whose error scales with the pixel's spread of luminance,
// not its level. The mean is L_r + sum(w d) / sum(w), kept as (hi, lo); the
// temporal gradient takes each consecutive pair's difference from its colour
// differences; the age weights, the time steps and the variance moments are
// FP32.
template <int CT, int G, int S>
__global__ void __launch_bounds__(256) k_pixel(int P, int b, float t_now, const uint32_t *__restrict__ state,
                                               const float *__restrict__ r_t, const uint32_t *__restrict__ r_seq,
                                               const void *__restrict__ r_col, float2 *__restrict__ lbar,
                                               float4 *__restrict__ pstat) {
    using CS = ColorStore<CT>;
    constexpr int L = G / S;
    const int l = threadIdx.x & (L - 1);
    const int groups = (gridDim.x * blockDim.x) / L;
    // every lane of a warp runs the same number of iterations (P rounded up)
    const int P_round = (P + (32 / L) - 1) / (32 / L) * (32 / L);
    for (int p = (blockIdx.x * blockDim.x + threadIdx.x) / L; p < P_round; p += groups) {
        const bool pix = p < P;
        const uint32_t st = pix ? __ldg(state + p) : 0u;
        const int n = (int)(st & 0xFFFFu), h = (int)(st >> 16);
        Entry E[S];
        float D[S];
#pragma unroll
        for (int r = 0; r < S; ++r) {
            const int k = r * L + l;
            E[r] = Entry{-INFINITY, 0.f, 0.f, 0.f, 0.f, 0u};
            if (k < n) {
                int s = h - 1 - k;
                if (s < 0) s += b;
                const size_t i = (size_t)p * b + s;
                E[r].T = __ldg(r_t + i);
                E[r].Q = __ldg(r_seq + i);
                const float3 c = CS::load(r_col, i);
                E[r].cx = c.x;
                E[r].cy = c.y;
                E[r].cz = c.z;
            }
        }
#pragma unroll
        for (int r = 0; r < S; ++r)
            if (r * L + l < n) E[r].w = expf(-kAgeDecay * fmaxf(t_now - E[r].T, 0.f));
        // reference: the newest sample (entry 0: lane 0, register 0)
        const float3 cr = make_float3(__shfl_sync(0xffffffffu, E[0].cx, 0, L),
                                      __shfl_sync(0xffffffffu, E[0].cy, 0, L),
                                      __shfl_sync(0xffffffffu, E[0].cz, 0, L));
        float lw = 0.f, lwd = 0.f;
#pragma unroll
        for (int r = 0; r < S; ++r) {   // L - L_r
            D[r] = r * L + l < n ? fmaf(kLumB, __fsub_rn(E[r].cz, cr.z),
                                        fmaf(kLumG, __fsub_rn(E[r].cy, cr.y), kLumR * __fsub_rn(E[r].cx, cr.x)))
                                 : 0.f;
            lw += E[r].w;
            lwd += E[r].w * D[r];
        }
        const float sw = group_sum<L>(lw);
        const float swd = group_sum<L>(lwd);
        const float delta = n > 0 ? swd / sw : 0.f;   // mean - L_r
        float lm2 = 0.f;
#pragma unroll
        for (int r = 0; r < S; ++r) {
            const float dd = r * L + l < n ? D[r] - delta : 0.f;
            lm2 += E[r].w * dd * dd;
        }
        const float m2 = group_sum<L>(lm2);
        // newest first by time, equal times newest first by sequence number;
        // queues filled in time order are already in that order
        float T[S], Tn[S];
        uint32_t Q[S], Qn[S];
#pragma unroll
        for (int r = 0; r < S; ++r) {
            T[r] = E[r].T;
            Q[r] = E[r].Q;
        }
        next_entry<L, S>(T, Tn, l);
        next_entry<L, S>(Q, Qn, l);
        bool ordered = true;
#pragma unroll
        for (int r = 0; r < S; ++r)
            ordered = ordered && (!(r * L + l + 1 < n) || (T[r] > Tn[r]) || (T[r] == Tn[r] && Q[r] > Qn[r]));
        if (!__all_sync(0xffffffffu, ordered)) {
            // bitonic sort of the group's G entries descending by (T, Q);
            // empty entries (-inf) sink. Entry e = r L + l: the partner at
            // distance j < L is in lane l ^ j, at j >= L in register r ^ (j / L)
            // of the same lane.
#pragma unroll
            for (int kk = 2; kk <= G; kk <<= 1) {
#pragma unroll
                for (int j = kk >> 1; j > 0; j >>= 1) {
                    if (j >= L) {
#pragma unroll
                        for (int r = 0; r < S; ++r) {
                            const int r2 = r ^ (j / L);
                            if (r2 < r) continue;   // each pair once, from its lower entry
                            const bool desc = ((r * L + l) & kk) == 0;
                            if (newer(E[r], E[r2]) != desc) {
                                const Entry t = E[r];
                                E[r] = E[r2];
                                E[r2] = t;
                            }
                        }
                        continue;
                    }
#pragma unroll
                    for (int r = 0; r < S; ++r) {
                        const int e = r * L + l;
                        Entry o;
                        o.T = __shfl_xor_sync(0xffffffffu, E[r].T, j, L);
                        o.Q = __shfl_xor_sync(0xffffffffu, E[r].Q, j, L);
                        o.cx = __shfl_xor_sync(0xffffffffu, E[r].cx, j, L);
                        o.cy = __shfl_xor_sync(0xffffffffu, E[r].cy, j, L);
                        o.cz = __shfl_xor_sync(0xffffffffu, E[r].cz, j, L);
                        o.w = __shfl_xor_sync(0xffffffffu, E[r].w, j, L);
                        const bool lower = (e & j) == 0, desc = (e & kk) == 0;
                        const bool keep = (lower == desc) ? newer(E[r], o) : !newer(E[r], o);
                        if (!keep) E[r] = o;
                    }
                }
            }
        }
        // consecutive luminance differences from the colour differences
        float cx[S], cy[S], cz[S], cxn[S], cyn[S], czn[S];
#pragma unroll
        for (int r = 0; r < S; ++r) {
            T[r] = E[r].T;
            cx[r] = E[r].cx;
            cy[r] = E[r].cy;
            cz[r] = E[r].cz;
        }
        next_entry<L, S>(cx, cxn, l);
        next_entry<L, S>(cy, cyn, l);
        next_entry<L, S>(cz, czn, l);
        next_entry<L, S>(T, Tn, l);
        float num = 0.f, den = 0.f;
#pragma unroll
        for (int r = 0; r < S; ++r) {
            if (r * L + l + 1 < n) {
                const float dL = fmaf(kLumB, __fsub_rn(cz[r], czn[r]),
                                      fmaf(kLumG, __fsub_rn(cy[r], cyn[r]), kLumR * __fsub_rn(cx[r], cxn[r])));
                num += E[r].w * fabsf(dL);
                den += E[r].w * (T[r] - Tn[r]);
            }
        }
        num = group_sum<L>(num);
        den = group_sum<L>(den);
        if (l == 0 && pix) {
            if (n == 0) {
                lbar[p] = make_float2(__int_as_float(0x7fc00000), 0.f);
                pstat[p] = make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                const dfloat Lr = luminance_df(cr);
                const dfloat mean = df_add(Lr, {delta, 0.f});
                const float gt = (n >= 2 && den > 0.f) ? num / den : 0.f;
                lbar[p] = make_float2(mean.h, mean.l);
                pstat[p] = make_float4(sw, mean.h, m2, gt);
            }
        }
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

// One block per statistics tile: G_x, G_y of each pixel from its neighbours'
// means (written to the gradient map) and the tile record: sample count,
// non-empty pixels, gradient sums, and the age-weighted luminance moments
// merged with Chan's formula (per thread and per warp in FP32, at most 2048
// samples each; across warps in FP64 once the tile holds more than 4096, the
// one FP64 step of the forward path). The record stores FP64 fields.
constexpr int kTileThreads = 256;

__global__ void __launch_bounds__(kTileThreads) k_spatial_tiles(int W, int H, int S, int ntx,
                                                                const float2 *__restrict__ lbar,
                                                                const float4 *__restrict__ pstat,
                                                                const uint32_t *__restrict__ state,
                                                                float4 *__restrict__ grad,
                                                                TilePartial *__restrict__ tiles) {
    const int tile = blockIdx.x;
    const int x0 = (tile % ntx) * S, y0 = (tile / ntx) * S;
    const int tw = min(S, W - x0), th = min(S, H - y0), A = tw * th;
    float n = 0.f, ne = 0.f, sgx = 0.f, sgy = 0.f, sgt = 0.f;
    Moments<float> mo{0.f, 0.f, 0.f};
    for (int k = threadIdx.x; k < A; k += blockDim.x) {
        const int x = x0 + k % tw, y = y0 + k / tw;
        const int p = y * W + x;
        const float2 lp = __ldg(lbar + p);
        const float l = lp.x;
        const float4 ps = __ldg(pstat + p);
        if (isnan(l)) {
            grad[p] = make_float4(0.f, 0.f, 0.f, l);
            continue;
        }
        // one-sided differences of the double-float means, rounded once
        float sx = 0.f, sy = 0.f;
        int mx = 0, my = 0;
        const dfloat lm = {lp.x, lp.y};
        float2 v;
        if (x > 0 && !isnan((v = __ldg(lbar + p - 1)).x)) { sx += fabsf(df_diff(lm, {v.x, v.y})); ++mx; }
        if (x + 1 < W && !isnan((v = __ldg(lbar + p + 1)).x)) { sx += fabsf(df_diff(lm, {v.x, v.y})); ++mx; }
        if (y > 0 && !isnan((v = __ldg(lbar + p - W)).x)) { sy += fabsf(df_diff(lm, {v.x, v.y})); ++my; }
        if (y + 1 < H && !isnan((v = __ldg(lbar + p + W)).x)) { sy += fabsf(df_diff(lm, {v.x, v.y})); ++my; }
        const float gx = mx ? sx / mx : 0.f, gy = my ? sy / my : 0.f;
        grad[p] = make_float4(gx, gy, ps.w, l);
        n += (float)(__ldg(state + p) & 0xFFFFu);
        ne += 1.f;
        sgx += gx;
        sgy += gy;
        sgt += ps.w;
        mo.merge(ps.x, ps.y, ps.z);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n += __shfl_xor_sync(0xffffffffu, n, o);
        ne += __shfl_xor_sync(0xffffffffu, ne, o);
        sgx += __shfl_xor_sync(0xffffffffu, sgx, o);
        sgy += __shfl_xor_sync(0xffffffffu, sgy, o);
        sgt += __shfl_xor_sync(0xffffffffu, sgt, o);
        const float w2 = __shfl_xor_sync(0xffffffffu, mo.w, o);
        const float mu2 = __shfl_xor_sync(0xffffffffu, mo.mean, o);
        const float s2 = __shfl_xor_sync(0xffffffffu, mo.m2, o);
        mo.merge(w2, mu2, s2);
    }
    __shared__ float sh[kTileThreads / 32][8];
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sh[warp][0] = n; sh[warp][1] = ne; sh[warp][2] = sgx; sh[warp][3] = sgy; sh[warp][4] = sgt;
        sh[warp][5] = mo.w; sh[warp][6] = mo.mean; sh[warp][7] = mo.m2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        TilePartial out;
        // FP32 across the warps: the counts are integers (exact below 2^24) and
        // the gradient sums add eight warp totals
        float tn = 0.f, tne = 0.f, tgx = 0.f, tgy = 0.f, tgt = 0.f;
        for (int w = 0; w < kTileThreads / 32; ++w) {
            tn += sh[w][0]; tne += sh[w][1]; tgx += sh[w][2]; tgy += sh[w][3]; tgt += sh[w][4];
        }
        if (tn > (float)kSortedBinMax) {   // more than 4096 samples: FP64 merge
            Moments<double> r{0.0, 0.0, 0.0};
            for (int w = 0; w < kTileThreads / 32; ++w) r.merge(sh[w][5], sh[w][6], sh[w][7]);
            out.sw = r.w; out.mean = r.mean; out.m2 = r.m2;
        } else {
            Moments<float> r{0.f, 0.f, 0.f};
            for (int w = 0; w < kTileThreads / 32; ++w) r.merge(sh[w][5], sh[w][6], sh[w][7]);
            out.sw = r.w; out.mean = r.mean; out.m2 = r.m2;
        }
        out.n = (uint32_t)tn;
        out.nonempty = (uint32_t)tne;
        out.sgx = tgx;
        out.sgy = tgy;
        out.sgt = tgt;
        out.pad[0] = out.pad[1] = out.pad[2] = 0u;
        tiles[tile] = out;
    }
}

// Queue entries per lane of the pixel pass.
constexpr int kPixelEntries = 4;

template <int CT>
cudaError_t launch_pixel(AfrContext *c, float t_now, cudaStream_t s) {
    constexpr int S = kPixelEntries;
    int g = grid_for((size_t)c->P * 32, 256, 16 * device_sms());
    if (c->b <= 4)
        k_pixel<CT, 4, 2><<<g, 256, 0, s>>>(c->P, c->b, t_now, c->r_state, c->r_t, c->r_seq, c->r_col, c->lbar,
                                            c->pstat);
    else if (c->b <= 8)
        k_pixel<CT, 8, S><<<g, 256, 0, s>>>(c->P, c->b, t_now, c->r_state, c->r_t, c->r_seq, c->r_col, c->lbar,
                                            c->pstat);
    else if (c->b <= 16)
        k_pixel<CT, 16, S><<<g, 256, 0, s>>>(c->P, c->b, t_now, c->r_state, c->r_t, c->r_seq, c->r_col, c->lbar,
                                             c->pstat);
    else
        k_pixel<CT, 32, S><<<g, 256, 0, s>>>(c->P, c->b, t_now, c->r_state, c->r_t, c->r_seq, c->r_col, c->lbar,
                                             c->pstat);
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
    k_spatial_tiles<<<c->ntiles, kTileThreads, 0, s>>>(c->W, c->H, c->S, c->ntx, c->lbar, c->pstat, c->r_state,
                                                      c->grad, c->tiles);
    return cudaGetLastError();
}

}  // namespace afr

// k_reproject.cu -- section 6.2: move every buffered sample to the display
// time along its screen velocity and rebin it into the frame view (a CSR
// over destination pixels).
//
//  count:   thread per queue slot; x' = x + m_x (t_now - t) with one rounding
//           per operation (__fmul_rn / __fadd_rn, so no contraction), drops
//           samples leaving the image, counts per destination bin (warp-
//           aggregated) and keeps the smallest a^2 per bin (the filter's
//           exponent shift).
//  scan:    bin offsets.
//  scatter: same slot walk, writes (x', y', a^2, seq) and the colour at the
//           bin's next free record.
//  order:   one warp per bin sorts its records by sequence number (a 32-lane
//           bitonic network, looped merges up to 4096 records) so that the
//           frame view, and every sum over it, is deterministic.
#include "afr_internal.cuh"

namespace afr {
namespace {

struct Moved {
    bool ok;
    uint32_t bin;
    float xp, yp, a2;
};

__device__ __forceinline__ Moved move_sample(float2 xy, float2 m, float t, float t_now, int W, int H) {
    Moved r;
    float a = __fsub_rn(t_now, t);
    r.xp = __fadd_rn(xy.x, __fmul_rn(m.x, a));
    r.yp = __fadd_rn(xy.y, __fmul_rn(m.y, a));
    r.a2 = __fmul_rn(a, a);
    r.ok = r.xp >= 0.f && r.xp < (float)W && r.yp >= 0.f && r.yp < (float)H;
    r.bin = r.ok ? (uint32_t)(int)floorf(r.yp) * (uint32_t)W + (uint32_t)(int)floorf(r.xp) : kInvalid;
    return r;
}

__device__ __forceinline__ bool slot_live(uint32_t st, int s, int b) {
    int n = (int)(st & 0xFFFFu), h = (int)(st >> 16);
    int age = h - 1 - s;
    if (age < 0) age += b;
    return age < n;
}

__global__ void __launch_bounds__(256) k_count(size_t nslots, int b, int W, int H, float t_now,
                                               const uint32_t *__restrict__ state, const float2 *__restrict__ r_xy,
                                               const float2 *__restrict__ r_mo, const float *__restrict__ r_t,
                                               uint32_t *__restrict__ fcnt, uint32_t *__restrict__ amin2,
                                               unsigned long long *__restrict__ dcount) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nslots; i += (size_t)gridDim.x * blockDim.x) {
        size_t p = i / b;
        int s = (int)(i - p * b);
        if (!slot_live(__ldg(state + p), s, b)) continue;
        Moved mv = move_sample(__ldg(r_xy + i), __ldg(r_mo + i), __ldg(r_t + i), t_now, W, H);
        agg_count(dcount + CNT_DROPPED, !mv.ok);
        if (!mv.ok) continue;
        agg_inc(fcnt, mv.bin);
        unsigned mask = __activemask();
        unsigned peers = __match_any_sync(mask, mv.bin);
        uint32_t bits = __reduce_min_sync(peers, __float_as_uint(mv.a2));   // a^2 >= 0: bit order = value order
        if ((threadIdx.x & 31) == __ffs(peers) - 1) atomicMin(amin2 + mv.bin, bits);
    }
}

template <int CT>
__global__ void __launch_bounds__(256) k_scatter(size_t nslots, int b, int W, int H, float t_now,
                                                 const uint32_t *__restrict__ state, const float2 *__restrict__ r_xy,
                                                 const float2 *__restrict__ r_mo, const float *__restrict__ r_t,
                                                 const uint32_t *__restrict__ r_seq, const void *__restrict__ r_col,
                                                 const uint32_t *__restrict__ foff, uint32_t *__restrict__ fcur,
                                                 float4 *__restrict__ fpos, void *__restrict__ fcol) {
    using CS = ColorStore<CT>;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nslots; i += (size_t)gridDim.x * blockDim.x) {
        size_t p = i / b;
        int s = (int)(i - p * b);
        if (!slot_live(__ldg(state + p), s, b)) continue;
        Moved mv = move_sample(__ldg(r_xy + i), __ldg(r_mo + i), __ldg(r_t + i), t_now, W, H);
        if (!mv.ok) continue;
        uint32_t e = __ldg(foff + mv.bin) + agg_inc(fcur, mv.bin);
        fpos[e] = make_float4(mv.xp, mv.yp, mv.a2, __uint_as_float(__ldg(r_seq + i)));
        reinterpret_cast<typename CS::T *>(fcol)[e] = CS::raw(r_col, i);
    }
}

// 64-bit keys (seq << 32 | record) sorted ascending across a warp
__device__ __forceinline__ unsigned long long warp_sort64(unsigned long long v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            unsigned long long o = __shfl_xor_sync(0xffffffffu, v, j);
            bool up = ((lane & k) == 0), lower = ((lane & j) == 0);
            v = (lower == up) ? (v < o ? v : o) : (v < o ? o : v);
        }
    }
    return v;
}

// Orders the records of each bin by sequence number. Bins with up to 32
// records sort in registers; larger bins (up to kSortedBinMax) are ranked by
// counting smaller sequence numbers, lane-parallel; larger ones stay in
// arrival order and are counted.
template <int CT>
__global__ void __launch_bounds__(256) k_order(int P, const uint32_t *__restrict__ foff,
                                               const float4 *__restrict__ src_pos, const void *__restrict__ src_col,
                                               float4 *__restrict__ dst_pos, void *__restrict__ dst_col,
                                               unsigned long long *__restrict__ dcount) {
    using CS = ColorStore<CT>;
    using T = typename CS::T;
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < P; q += warps) {
        uint32_t beg = __ldg(foff + q), m = __ldg(foff + q + 1) - beg;
        if (m == 0) continue;
        if (m <= 32) {
            unsigned long long key = ~0ull;
            if (lane < (int)m) key = ((unsigned long long)__float_as_uint(src_pos[beg + lane].w) << 32) | (beg + lane);
            key = warp_sort64(key);
            if (lane < (int)m) {
                uint32_t from = (uint32_t)key;
                dst_pos[beg + lane] = src_pos[from];
                reinterpret_cast<T *>(dst_col)[beg + lane] = CS::raw(src_col, from);
            }
        } else if (m <= (uint32_t)kSortedBinMax) {
            for (uint32_t j = lane; j < m; j += 32) {
                uint32_t sj = __float_as_uint(src_pos[beg + j].w);
                uint32_t rank = 0;
                for (uint32_t k = 0; k < m; ++k) rank += __float_as_uint(src_pos[beg + k].w) < sj;
                dst_pos[beg + rank] = src_pos[beg + j];
                reinterpret_cast<T *>(dst_col)[beg + rank] = CS::raw(src_col, beg + j);
            }
        } else {
            for (uint32_t j = lane; j < m; j += 32) {
                dst_pos[beg + j] = src_pos[beg + j];
                reinterpret_cast<T *>(dst_col)[beg + j] = CS::raw(src_col, beg + j);
            }
            if (lane == 0) atomicAdd(dcount + CNT_UNSORTED, 1ull);
        }
    }
}

__global__ void k_fill_u32(uint32_t *p, size_t n, uint32_t v) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

}  // namespace

cudaError_t launch_reproject(AfrContext *c, float t_now, cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(c->fcnt, 0, sizeof(uint32_t) * c->P, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->dcount + CNT_DROPPED, 0, sizeof(unsigned long long) * 2, s)) != cudaSuccess) return e;
    k_fill_u32<<<grid_for(c->P, 256), 256, 0, s>>>(c->amin2, c->P, 0x7f800000u);
    int g = grid_for(c->nslots, 256);
    k_count<<<g, 256, 0, s>>>(c->nslots, c->b, c->W, c->H, t_now, c->r_state, c->r_xy, c->r_mo, c->r_t, c->fcnt,
                              c->amin2, c->dcount);
    if ((e = scan_exclusive(c->fcnt, c->foff, c->P, c->scan_tmp, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->fcnt, 0, sizeof(uint32_t) * c->P, s)) != cudaSuccess) return e;
    // records land unordered in the second half of the buffers, then k_order
    // writes them ordered into the first half
    float4 *tmp_pos = c->fpos + c->frame_cap;
    void *tmp_col = static_cast<char *>(c->fcol) + c->frame_cap * c->csize;
    int go = grid_for((size_t)c->P * 32, 256);
    switch (c->ct) {
        case AFR_F32:
            k_scatter<AFR_F32><<<g, 256, 0, s>>>(c->nslots, c->b, c->W, c->H, t_now, c->r_state, c->r_xy, c->r_mo, c->r_t,
                                                 c->r_seq, c->r_col, c->foff, c->fcnt, tmp_pos, tmp_col);
            k_order<AFR_F32><<<go, 256, 0, s>>>(c->P, c->foff, tmp_pos, tmp_col, c->fpos, c->fcol, c->dcount);
            break;
        case AFR_F16:
            k_scatter<AFR_F16><<<g, 256, 0, s>>>(c->nslots, c->b, c->W, c->H, t_now, c->r_state, c->r_xy, c->r_mo, c->r_t,
                                                 c->r_seq, c->r_col, c->foff, c->fcnt, tmp_pos, tmp_col);
            k_order<AFR_F16><<<go, 256, 0, s>>>(c->P, c->foff, tmp_pos, tmp_col, c->fpos, c->fcol, c->dcount);
            break;
        default:
            k_scatter<AFR_BF16><<<g, 256, 0, s>>>(c->nslots, c->b, c->W, c->H, t_now, c->r_state, c->r_xy, c->r_mo, c->r_t,
                                                  c->r_seq, c->r_col, c->foff, c->fcnt, tmp_pos, tmp_col);
            k_order<AFR_BF16><<<go, 256, 0, s>>>(c->P, c->foff, tmp_pos, tmp_col, c->fpos, c->fcol, c->dcount);
            break;
    }
    return cudaGetLastError();
}

}  // namespace afr

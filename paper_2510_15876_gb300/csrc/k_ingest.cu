// k_ingest.cu -- section 4 deep buffer: counting-sort a batch of samples by
// pixel and push each pixel's share into its queue of depth b.
//
//  1. hist:    validate each sample, record its pixel and its ticket (its
//              rank among the pixel's samples in atomic order; warp-
//              aggregated atomics: lanes hitting one pixel share one), and repack the sample into one aligned record (48 B for FP32
//              colours, 32 B for 16-bit) so that the commit gathers one
//              record instead of three scattered fields.
//  2. scan:    pixel offsets of the batch's counting sort.
//  3. scatter: write each sample's batch index into its pixel's segment at
//              offset + ticket (no atomics).
//  4. commit:  one warp per pixel sorts the segment's indices (= insertion
//              order) with a 32-lane bitonic network, keeps the min(b, m)
//              newest, and writes them into the circular queue at
//              (head + rank) mod b, the slots sequential pushes would use.
#include "afr_internal.cuh"

namespace afr {
namespace {

// Packed sample: a = (x, y, t, depth); colour and motion follow (layout per type).
template <int CT> struct Packed;
template <> struct Packed<AFR_F32> {
    float4 a, b, c;   // b = (r, g, b, mx), c = (my, -, -, -)
    static __device__ __forceinline__ void store(Packed *dst, float4 p, float4 col, float2 m) {
        dst->a = p;
        dst->b = make_float4(col.x, col.y, col.z, m.x);
        dst->c = make_float4(m.y, 0.f, 0.f, 0.f);
    }
    __device__ __forceinline__ float4 color() const { return make_float4(b.x, b.y, b.z, 0.f); }
    __device__ __forceinline__ float2 motion() const { return make_float2(b.w, c.x); }
};
struct Packed16 {
    float4 a;
    uint4 b;          // (r | g << 16, b, mx bits, my bits)
    static __device__ __forceinline__ void store(Packed16 *dst, float4 p, ushort4 col, float2 m) {
        dst->a = p;
        dst->b = make_uint4((uint32_t)col.x | ((uint32_t)col.y << 16), (uint32_t)col.z, __float_as_uint(m.x),
                            __float_as_uint(m.y));
    }
    __device__ __forceinline__ ushort4 color() const {
        return make_ushort4((unsigned short)(b.x & 0xFFFFu), (unsigned short)(b.x >> 16), (unsigned short)b.y, 0);
    }
    __device__ __forceinline__ float2 motion() const { return make_float2(__uint_as_float(b.z), __uint_as_float(b.w)); }
};
template <> struct Packed<AFR_F16> : Packed16 {};
template <> struct Packed<AFR_BF16> : Packed16 {};

template <int CT>
__global__ void __launch_bounds__(256) k_hist(const float4 *__restrict__ pos, const void *__restrict__ col,
                                              const float2 *__restrict__ mo, uint32_t n, int W, int H,
                                              uint2 *__restrict__ bin_of, uint32_t *__restrict__ pcnt,
                                              Packed<CT> *__restrict__ pk, unsigned long long *__restrict__ dcount) {
    using CS = ColorStore<CT>;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float4 p = __ldg(pos + i);
        typename CS::T cr = CS::raw(col, i);
        float3 c = CS::widen(cr);
        float2 m = __ldg(mo + i);
        bool ok = isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && isfinite(c.x) && isfinite(c.y) &&
                  isfinite(c.z) && isfinite(m.x) && isfinite(m.y) && p.x >= 0.f && p.y >= 0.f &&
                  p.x < (float)W && p.y < (float)H;
        uint2 bt = make_uint2(kInvalid, 0u);
        if (ok) {
            bt.x = (uint32_t)(int)floorf(p.y) * (uint32_t)W + (uint32_t)(int)floorf(p.x);
            Packed<CT>::store(pk + i, p, cr, m);
            bt.y = agg_inc(pcnt, bt.x);
        }
        bin_of[i] = bt;
        agg_count(dcount + CNT_REJECTED, !ok);
    }
}

__global__ void __launch_bounds__(256) k_scatter(const uint2 *__restrict__ bin_of, uint32_t n,
                                                 const uint32_t *__restrict__ poff, uint32_t *__restrict__ idx) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint2 bt = bin_of[i];
        if (bt.x == kInvalid) continue;
        idx[__ldg(poff + bt.x) + bt.y] = i;
    }
}

// ascending bitonic sort of one key per lane across a full warp
__device__ __forceinline__ uint32_t warp_sort_asc(uint32_t v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            uint32_t o = __shfl_xor_sync(0xffffffffu, v, j);
            bool up = ((lane & k) == 0);
            bool lower = ((lane & j) == 0);
            v = (lower == up) ? min(v, o) : max(v, o);
        }
    }
    return v;
}

// merge step of a bitonic sequence held across the warp into ascending order
__device__ __forceinline__ uint32_t warp_merge_asc(uint32_t v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        uint32_t o = __shfl_xor_sync(0xffffffffu, v, j);
        v = ((lane & j) == 0) ? min(v, o) : max(v, o);
    }
    return v;
}

template <int CT>
__global__ void __launch_bounds__(256) k_commit(const uint32_t *__restrict__ poff, const uint32_t *__restrict__ idx,
                                                int P, int b, uint32_t seq0, const Packed<CT> *__restrict__ pk,
                                                float2 *__restrict__ r_xy, float2 *__restrict__ r_mo,
                                                float *__restrict__ r_t, float *__restrict__ r_depth,
                                                uint32_t *__restrict__ r_seq, void *__restrict__ r_col,
                                                uint32_t *__restrict__ r_state) {
    using CS = ColorStore<CT>;
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < P; p += warps) {
        uint32_t beg = poff[p], m = poff[p + 1] - beg;
        if (m == 0) continue;
        // keys are batch index + 1; 0 marks an empty lane and sorts first
        uint32_t key = lane < (int)m ? idx[beg + lane] + 1u : 0u;
        key = warp_sort_asc(key);
        for (uint32_t c = 32; c < m; c += 32) {
            uint32_t k2 = c + lane < m ? idx[beg + c + lane] + 1u : 0u;
            k2 = warp_sort_asc(k2);
            uint32_t rev = __shfl_sync(0xffffffffu, k2, 31 - lane);
            key = warp_merge_asc(max(key, rev));   // the 32 largest so far, ascending
        }
        uint32_t st = r_state[p];
        uint32_t c0 = st & 0xFFFFu, h0 = st >> 16;
        uint32_t kept = m < (uint32_t)b ? m : (uint32_t)b;
        if (lane >= 32 - (int)kept) {
            uint32_t i = key - 1u;
            uint32_t rank = m - 32u + (uint32_t)lane;           // position in insertion order
            uint32_t s = (h0 + rank) % (uint32_t)b;
            size_t dst = (size_t)p * b + s;
            const Packed<CT> rec = pk[i];
            r_xy[dst] = make_float2(rec.a.x, rec.a.y);
            r_t[dst] = rec.a.z;
            r_depth[dst] = rec.a.w;
            r_mo[dst] = rec.motion();
            r_seq[dst] = seq0 + i;
            reinterpret_cast<typename CS::T *>(r_col)[dst] = rec.color();
        }
        if (lane == 0) {
            uint32_t cn = (uint64_t)c0 + m < (uint64_t)b ? c0 + m : (uint32_t)b;
            uint32_t hn = (uint32_t)((h0 + (uint64_t)m) % (uint32_t)b);
            r_state[p] = cn | (hn << 16);
        }
    }
}

template <int CT>
cudaError_t run(AfrContext *c, const float4 *pos, const void *col, const float2 *mo, uint32_t n, uint32_t seq0,
                cudaStream_t s) {
    Packed<CT> *pk = reinterpret_cast<Packed<CT> *>(c->pack);
    cudaError_t e = cudaMemsetAsync(c->pcnt, 0, sizeof(uint32_t) * c->P, s);
    if (e != cudaSuccess) return e;
    int g = grid_for(n, 256);
    k_hist<CT><<<g, 256, 0, s>>>(pos, col, mo, n, c->W, c->H, c->bin_of, c->pcnt, pk, c->dcount);
    if ((e = scan_exclusive(c->pcnt, c->poff, c->P, c->scan_tmp, s)) != cudaSuccess) return e;
    k_scatter<<<g, 256, 0, s>>>(c->bin_of, n, c->poff, c->idx);
    int gc = grid_for((size_t)c->P * 32, 256);
    k_commit<CT><<<gc, 256, 0, s>>>(c->poff, c->idx, c->P, c->b, seq0, pk, c->r_xy, c->r_mo, c->r_t, c->r_depth,
                                    c->r_seq, c->r_col, c->r_state);
    return cudaGetLastError();
}

}  // namespace

size_t packed_bytes(int ct) { return ct == AFR_F32 ? sizeof(Packed<AFR_F32>) : sizeof(Packed16); }

cudaError_t launch_ingest(AfrContext *c, const AfrSampleBatch *batch, uint32_t n, uint32_t seq0,
                          cudaStream_t s) {
    const float4 *pos = reinterpret_cast<const float4 *>(batch->pos_dev);
    const float2 *mo = reinterpret_cast<const float2 *>(batch->motion_dev);
    const void *col = batch->color_dev;
    switch (c->ct) {
        case AFR_F32: return run<AFR_F32>(c, pos, col, mo, n, seq0, s);
        case AFR_F16: return run<AFR_F16>(c, pos, col, mo, n, seq0, s);
        default: return run<AFR_BF16>(c, pos, col, mo, n, seq0, s);
    }
}

}  // namespace afr

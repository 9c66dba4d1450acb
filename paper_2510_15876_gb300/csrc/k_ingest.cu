// k_ingest.cu -- section 4 deep buffer: counting-sort a batch of samples by
// pixel and push each pixel's share into its queue of depth b.
//
//  1. hist:   validate each sample, record its pixel and its ticket (its rank
//             among the pixel's samples in atomic order).
//  2. scan:   pixel offsets of the counting sort.
//  3. place:  write each sample, repacked into one 64-byte record that also
//             carries its batch index, at offset + ticket. A warp stages its
//             32 records in shared memory and stores them back four lanes per
//             record, so every record is one whole 64-byte block (no partial
//             sectors for the memory system to merge).
//  4. commit: one warp per pixel reads the pixel's records (contiguous),
//             ranks them by batch index (= insertion order): up to 32 records
//             by counting smaller indices across the warp, more by a chunked
//             bitonic top-32; keeps the min(b, m) newest and writes them into
//             the circular queue at (head + rank) mod b, the slots sequential
//             pushes would use.
#include "afr_internal.cuh"

namespace afr {
namespace {

// 64-byte staging record: a = (x, y, t, depth); b = colour and motion;
// c.y = batch index. F32: b = (r, g, b, m_x), c.x = m_y. 16-bit colours:
// b = (r | g << 16, b, m_x, m_y).
struct alignas(64) Rec64 {
    uint4 a, b, c, d;
};

template <int CT> struct RecCodec;
template <> struct RecCodec<AFR_F32> {
    using T = float4;
    static __device__ __forceinline__ void pack(Rec64 &r, float4 p, T col, float2 m, uint32_t i) {
        r.a = make_uint4(__float_as_uint(p.x), __float_as_uint(p.y), __float_as_uint(p.z), __float_as_uint(p.w));
        r.b = make_uint4(__float_as_uint(col.x), __float_as_uint(col.y), __float_as_uint(col.z),
                         __float_as_uint(m.x));
        r.c = make_uint4(__float_as_uint(m.y), i, 0u, 0u);
        r.d = make_uint4(0u, 0u, 0u, 0u);
    }
    static __device__ __forceinline__ T color(uint4 b, uint4) {
        return make_float4(__uint_as_float(b.x), __uint_as_float(b.y), __uint_as_float(b.z), 0.f);
    }
    static __device__ __forceinline__ float2 motion(uint4 b, uint4 c) {
        return make_float2(__uint_as_float(b.w), __uint_as_float(c.x));
    }
};
struct RecCodec16 {
    using T = ushort4;
    static __device__ __forceinline__ void pack(Rec64 &r, float4 p, T col, float2 m, uint32_t i) {
        r.a = make_uint4(__float_as_uint(p.x), __float_as_uint(p.y), __float_as_uint(p.z), __float_as_uint(p.w));
        r.b = make_uint4((uint32_t)col.x | ((uint32_t)col.y << 16), (uint32_t)col.z, __float_as_uint(m.x),
                         __float_as_uint(m.y));
        r.c = make_uint4(0u, i, 0u, 0u);
        r.d = make_uint4(0u, 0u, 0u, 0u);
    }
    static __device__ __forceinline__ T color(uint4 b, uint4) {
        return make_ushort4((unsigned short)(b.x & 0xFFFFu), (unsigned short)(b.x >> 16), (unsigned short)b.y, 0);
    }
    static __device__ __forceinline__ float2 motion(uint4 b, uint4) {
        return make_float2(__uint_as_float(b.z), __uint_as_float(b.w));
    }
};
template <> struct RecCodec<AFR_F16> : RecCodec16 {};
template <> struct RecCodec<AFR_BF16> : RecCodec16 {};

template <int CT>
__global__ void __launch_bounds__(256) k_hist(const float4 *__restrict__ pos, const void *__restrict__ col,
                                              const float2 *__restrict__ mo, uint32_t n, int W, int H,
                                              uint2 *__restrict__ bin_of, uint32_t *__restrict__ pcnt,
                                              unsigned long long *__restrict__ dcount) {
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
            bt.y = atomicAdd(pcnt + bt.x, 1u);   // a batch in time order rarely repeats a pixel within a warp
        }
        bin_of[i] = bt;
        agg_count(dcount + CNT_REJECTED, !ok);
    }
}

// Each warp takes 32 consecutive samples: lanes build their records in
// shared memory (80-byte stride: conflict-free 16-byte accesses), then lane
// 4k + q stores part q of record 8r + k in round r.
constexpr int kPlaceWarps = 8;

template <int CT>
__global__ void __launch_bounds__(32 * kPlaceWarps) k_place(const float4 *__restrict__ pos,
                                                            const void *__restrict__ col,
                                                            const float2 *__restrict__ mo, uint32_t n,
                                                            const uint2 *__restrict__ bin_of,
                                                            const uint32_t *__restrict__ poff,
                                                            const float4 *__restrict__ world,
                                                            Rec64 *__restrict__ pk) {
    using CS = ColorStore<CT>;
    __shared__ uint4 stage[kPlaceWarps][32][5];
    __shared__ uint32_t dest[kPlaceWarps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t nwarps = gridDim.x * kPlaceWarps;
    for (uint32_t base = (blockIdx.x * kPlaceWarps + w) * 32u; base < n; base += nwarps * 32u) {
        const uint32_t i = base + lane;
        uint32_t d = kInvalid;
        if (i < n) {
            const uint2 bt = bin_of[i];
            if (bt.x != kInvalid) {
                d = __ldg(poff + bt.x) + bt.y;
                Rec64 r;
                RecCodec<CT>::pack(r, __ldg(pos + i), CS::raw(col, i), __ldg(mo + i), i);
                if (world) {   // hit point in the record's spare 16 bytes
                    const float4 w = __ldg(world + i);
                    r.d = make_uint4(__float_as_uint(w.x), __float_as_uint(w.y), __float_as_uint(w.z), 0u);
                }
                stage[w][lane][0] = r.a;
                stage[w][lane][1] = r.b;
                stage[w][lane][2] = r.c;
                stage[w][lane][3] = r.d;
            }
        }
        dest[w][lane] = d;
        __syncwarp();
#pragma unroll
        for (int round = 0; round < 4; ++round) {
            const int k = round * 8 + (lane >> 2), q = lane & 3;
            const uint32_t dk = dest[w][k];
            if (dk != kInvalid) reinterpret_cast<uint4 *>(pk + dk)[q] = stage[w][k][q];
        }
        __syncwarp();
    }
}

// ascending bitonic sort of one 64-bit key per lane across a full warp
__device__ __forceinline__ unsigned long long warp_sort_asc(unsigned long long v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            unsigned long long o = __shfl_xor_sync(0xffffffffu, v, j);
            bool up = ((lane & k) == 0);
            bool lower = ((lane & j) == 0);
            v = (lower == up) ? min(v, o) : max(v, o);
        }
    }
    return v;
}

// merge step of a bitonic sequence held across the warp into ascending order
__device__ __forceinline__ unsigned long long warp_merge_asc(unsigned long long v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        unsigned long long o = __shfl_xor_sync(0xffffffffu, v, j);
        v = ((lane & j) == 0) ? min(v, o) : max(v, o);
    }
    return v;
}

// sort key of record e of a pixel's segment: (batch index + 1) << 32 | position
__device__ __forceinline__ unsigned long long rec_key(const Rec64 *__restrict__ pk, uint32_t beg, uint32_t e) {
    const uint32_t i = __ldg(&pk[beg + e].c.y);
    return ((unsigned long long)(i + 1u) << 32) | e;
}

template <int CT>
__global__ void __launch_bounds__(256) k_commit(const uint32_t *__restrict__ poff, int P, int b, uint32_t seq0,
                                                const Rec64 *__restrict__ pk, float2 *__restrict__ r_xy,
                                                float2 *__restrict__ r_mo, float *__restrict__ r_t,
                                                float *__restrict__ r_depth, uint32_t *__restrict__ r_seq,
                                                void *__restrict__ r_col, uint32_t *__restrict__ r_state,
                                                float4 *__restrict__ r_world) {
    using Codec = RecCodec<CT>;
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); p < P; p += warps) {
        const uint32_t beg = poff[p], m = poff[p + 1] - beg;
        if (m == 0) continue;
        const uint32_t st = r_state[p];
        const uint32_t c0 = st & 0xFFFFu, h0 = st >> 16;
        const uint32_t kept = m < (uint32_t)b ? m : (uint32_t)b;
        if (lane == 0) {
            const uint32_t cn = (uint64_t)c0 + m < (uint64_t)b ? c0 + m : (uint32_t)b;
            const uint32_t hn = (uint32_t)((h0 + (uint64_t)m) % (uint32_t)b);
            r_state[p] = cn | (hn << 16);
        }
        if (m <= 32) {
            // lane k holds record k; its rank in insertion order is the number
            // of the pixel's records with a smaller batch index (indices are unique)
            Rec64 rec;
            uint32_t i = 0xFFFFFFFFu;
            if (lane < (int)m) {
                rec.a = __ldg(&pk[beg + lane].a);
                rec.b = __ldg(&pk[beg + lane].b);
                rec.c = __ldg(&pk[beg + lane].c);
                i = rec.c.y;
            }
            uint32_t rank = 0;
            for (uint32_t k = 0; k < m; ++k) rank += __shfl_sync(0xffffffffu, i, k) < i;
            if (lane < (int)m && rank >= m - kept) {
                const uint32_t s = (h0 + rank) % (uint32_t)b;
                const size_t dst = (size_t)p * b + s;
                r_xy[dst] = make_float2(__uint_as_float(rec.a.x), __uint_as_float(rec.a.y));
                r_t[dst] = __uint_as_float(rec.a.z);
                r_depth[dst] = __uint_as_float(rec.a.w);
                r_mo[dst] = Codec::motion(rec.b, rec.c);
                r_seq[dst] = seq0 + i;
                reinterpret_cast<typename Codec::T *>(r_col)[dst] = Codec::color(rec.b, rec.c);
                if (r_world) {
                    const uint4 d = __ldg(&pk[beg + lane].d);
                    r_world[dst] = make_float4(__uint_as_float(d.x), __uint_as_float(d.y), __uint_as_float(d.z), 0.f);
                }
            }
            continue;
        }
        // more than 32: the 32 newest by chunked bitonic top-32 (0 marks an
        // empty lane and sorts first)
        unsigned long long key = lane < (int)m ? rec_key(pk, beg, lane) : 0ull;
        key = warp_sort_asc(key);
        for (uint32_t c = 32; c < m; c += 32) {
            unsigned long long k2 = c + lane < m ? rec_key(pk, beg, c + lane) : 0ull;
            k2 = warp_sort_asc(k2);
            const unsigned long long rev = __shfl_sync(0xffffffffu, k2, 31 - lane);
            key = warp_merge_asc(max(key, rev));   // the 32 largest so far, ascending
        }
        if (lane >= 32 - (int)kept) {
            const uint32_t i = (uint32_t)(key >> 32) - 1u;
            const Rec64 &rec = pk[beg + (uint32_t)key];
            const uint4 ra = rec.a, rb = rec.b, rc = rec.c;
            const uint32_t rank = m - 32u + (uint32_t)lane;           // position in insertion order
            const uint32_t s = (h0 + rank) % (uint32_t)b;
            const size_t dst = (size_t)p * b + s;
            r_xy[dst] = make_float2(__uint_as_float(ra.x), __uint_as_float(ra.y));
            r_t[dst] = __uint_as_float(ra.z);
            r_depth[dst] = __uint_as_float(ra.w);
            r_mo[dst] = Codec::motion(rb, rc);
            r_seq[dst] = seq0 + i;
            reinterpret_cast<typename Codec::T *>(r_col)[dst] = Codec::color(rb, rc);
            if (r_world) {
                const uint4 d = rec.d;
                r_world[dst] = make_float4(__uint_as_float(d.x), __uint_as_float(d.y), __uint_as_float(d.z), 0.f);
            }
        }
    }
}

template <int CT>
cudaError_t run(AfrContext *c, const float4 *pos, const void *col, const float2 *mo, const float4 *world, uint32_t n,
                uint32_t seq0, cudaStream_t s) {
    Rec64 *pk = reinterpret_cast<Rec64 *>(c->pack);
    cudaError_t e = cudaMemsetAsync(c->pcnt, 0, sizeof(uint32_t) * c->P, s);
    if (e != cudaSuccess) return e;
    const int g = grid_for(n, 256);
    k_hist<CT><<<g, 256, 0, s>>>(pos, col, mo, n, c->W, c->H, c->bin_of, c->pcnt, c->dcount);
    if ((e = scan_exclusive(c->pcnt, c->poff, c->P, c->scan_tmp, s)) != cudaSuccess) return e;
    k_place<CT><<<grid_for(n, 32 * kPlaceWarps), 32 * kPlaceWarps, 0, s>>>(pos, col, mo, n, c->bin_of, c->poff,
                                                                          c->r_world ? world : nullptr, pk);
    const int gc = grid_for((size_t)c->P * 32, 256);
    k_commit<CT><<<gc, 256, 0, s>>>(c->poff, c->P, c->b, seq0, pk, c->r_xy, c->r_mo, c->r_t, c->r_depth, c->r_seq,
                                    c->r_col, c->r_state, c->r_world);
    return cudaGetLastError();
}

// ---- reconstructor queue (section 5.2) ----------------------------------------
// The batch's accepted samples (k_hist marked the rejected ones) enter the
// N-slot queue in index order: a scan gives each its rank r among the
// batch's accepted samples, and it lands at slot (total + r) mod N; of a batch
// with more than N accepted samples only the last N are written.
__global__ void __launch_bounds__(256) k_fifo_flag(const uint2 *__restrict__ bin_of, uint32_t n,
                                                   uint32_t *__restrict__ flag) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        flag[i] = bin_of[i].x != kInvalid ? 1u : 0u;
}

template <int CT>
__global__ void __launch_bounds__(256) k_fifo_append(const float4 *__restrict__ pos, const void *__restrict__ col,
                                                     const float2 *__restrict__ mo, uint32_t n,
                                                     const uint32_t *__restrict__ flag,
                                                     const uint32_t *__restrict__ rank, uint32_t seq0, uint32_t N,
                                                     const uint32_t *__restrict__ total, float2 *__restrict__ q_xy,
                                                     float2 *__restrict__ q_mo, float *__restrict__ q_t,
                                                     uint32_t *__restrict__ q_seq, void *__restrict__ q_col,
                                                     const float4 *__restrict__ world, float4 *__restrict__ q_world) {
    using CS = ColorStore<CT>;
    const uint32_t accepted = rank[n - 1] + flag[n - 1], t0 = *total;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (!flag[i] || (uint64_t)rank[i] + N < accepted) continue;
        const uint32_t k = (uint32_t)(((uint64_t)t0 + rank[i]) % N);
        const float4 p = __ldg(pos + i);
        q_xy[k] = make_float2(p.x, p.y);
        q_t[k] = p.z;
        q_mo[k] = __ldg(mo + i);
        q_seq[k] = seq0 + i;
        reinterpret_cast<typename CS::T *>(q_col)[k] = CS::raw(col, i);
        if (q_world) {
            const float4 w = __ldg(world + i);
            q_world[k] = make_float4(w.x, w.y, w.z, 0.f);
        }
    }
}

__global__ void k_fifo_advance(const uint32_t *__restrict__ flag, const uint32_t *__restrict__ rank, uint32_t n,
                               uint32_t *__restrict__ total) {
    *total += rank[n - 1] + flag[n - 1];
}

template <int CT>
cudaError_t run_fifo(AfrContext *c, const float4 *pos, const void *col, const float2 *mo, const float4 *world,
                     uint32_t n, uint32_t seq0, cudaStream_t s) {
    const int g = grid_for(n, 256);
    k_fifo_flag<<<g, 256, 0, s>>>(c->bin_of, n, c->fifo_flag);
    cudaError_t e = scan_exclusive(c->fifo_flag, c->fifo_rank, n, c->fifo_scan, s);
    if (e != cudaSuccess) return e;
    k_fifo_append<CT><<<g, 256, 0, s>>>(pos, col, mo, n, c->fifo_flag, c->fifo_rank, seq0, (uint32_t)c->fifo_n,
                                        c->q_total, c->q_xy, c->q_mo, c->q_t, c->q_seq, c->q_col, world,
                                        c->q_world);
    k_fifo_advance<<<1, 1, 0, s>>>(c->fifo_flag, c->fifo_rank, n, c->q_total);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_fifo_append(AfrContext *c, const AfrSampleBatch *batch, uint32_t n, uint32_t seq0,
                               cudaStream_t s) {
    const float4 *pos = reinterpret_cast<const float4 *>(batch->pos_dev);
    const float2 *mo = reinterpret_cast<const float2 *>(batch->motion_dev);
    const float4 *world = reinterpret_cast<const float4 *>(batch->world_dev);
    switch (c->ct) {
        case AFR_F32: return run_fifo<AFR_F32>(c, pos, batch->color_dev, mo, world, n, seq0, s);
        case AFR_F16: return run_fifo<AFR_F16>(c, pos, batch->color_dev, mo, world, n, seq0, s);
        default: return run_fifo<AFR_BF16>(c, pos, batch->color_dev, mo, world, n, seq0, s);
    }
}

size_t packed_bytes(int) { return sizeof(Rec64); }

cudaError_t launch_ingest(AfrContext *c, const AfrSampleBatch *batch, uint32_t n, uint32_t seq0,
                          cudaStream_t s) {
    const float4 *pos = reinterpret_cast<const float4 *>(batch->pos_dev);
    const float2 *mo = reinterpret_cast<const float2 *>(batch->motion_dev);
    const void *col = batch->color_dev;
    const float4 *world = reinterpret_cast<const float4 *>(batch->world_dev);
    switch (c->ct) {
        case AFR_F32: return run<AFR_F32>(c, pos, col, mo, world, n, seq0, s);
        case AFR_F16: return run<AFR_F16>(c, pos, col, mo, world, n, seq0, s);
        default: return run<AFR_BF16>(c, pos, col, mo, world, n, seq0, s);
    }
}

}  // namespace afr

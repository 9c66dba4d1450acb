// k_ingest.cu -- section 4 deep buffer: push a batch of samples into the
// per-pixel queues of depth b (each keeps its b newest samples by insertion
// order).
//
// The batch arrives in insertion order with its samples spread over the whole
// image, and the queues are planes in pixel order, so ingest is a counting
// sort by pixel followed by a per-pixel selection:
//
//  1. count:   per pixel, the samples whose position is valid (reads only the
//              16-byte position of each sample).
//  2. scan:    bucket offsets, one bucket per pixel.
//  3. scatter: each sample appends its 64-byte record (position, colour,
//              motion, batch index, hit point) to its pixel's bucket. A warp
//              stages its 32 records in shared memory and stores each with
//              four lanes, so every store is two whole sectors. The pixel's
//              append cursor starts at the bucket's offset, so the ticket its
//              atomic returns is the record's place; a thread takes the tickets
//              of both its samples before using either. A sample whose colour
//              or motion is not finite leaves a dead record (batch index
//              kInvalid).
//  4. commit:  a thread per bucket record, in bucket (= pixel) order: its
//              rank among its pixel's live records is the number of them with
//              a smaller batch index (read from shared memory, where a block
//              keeps the batch indices of the records it holds); the newest
//              min(b, m) go to the queue slots
//              (head + rank) mod b that sequential pushes would use, so a
//              warp's stores cover consecutive slots. The first record of each
//              pixel writes the pixel's new queue state (from a copy of the
//              states taken before the commit, which every thread reads). A
//              pixel with more than kBigPixel records is left to a warp that
//              streams its bucket keeping the newest 32 in registers.
#include "afr_internal.cuh"

namespace afr {
namespace {

constexpr uint32_t kBigPixel = 256;   // records of one pixel above which a warp selects the newest b

// Bucket records, 4 uint4 (64 bytes: two whole sectors) each:
//   q0 = (x, y, t, batch index)
//   q1 = FP32: (r, g, b, m_x); 16-bit: (r | g << 16, b, m_x, m_y)
//   q2 = (m_y for FP32 colours, depth, hit point X, Y)
//   q3 = (hit point Z, 0, 0, 0)
// (Three-part, 48-byte records, whose halves of a shared sector L2 has to
// merge, measured slower.)
constexpr int NP = 4;
struct Bucket {
    uint4 *r;    // [NP * batch_cap]
};

// Destination planes of the queues (slot p * b + s).
struct Queues {
    float2 *xy, *mo;
    float *t, *depth;
    uint32_t *seq;
    void *col;
    uint32_t *state;   // count | head << 16
    float4 *world;
    size_t nslots;     // P * b (checks)
};

__device__ __forceinline__ bool position_ok(float4 p, int W, int H) {
    return isfinite(p.x) && isfinite(p.y) && isfinite(p.z) && p.x >= 0.f && p.y >= 0.f && p.x < (float)W &&
           p.y < (float)H;
}

__device__ __forceinline__ uint32_t pixel_at(float x, float y, int W) {
    return (uint32_t)(int)floorf(y) * (uint32_t)W + (uint32_t)(int)floorf(x);
}

__global__ void __launch_bounds__(256) k_pix_count(const float4 *__restrict__ pos, uint32_t n, int W, int H,
                                                   uint32_t *__restrict__ pcnt) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 p = __ldg(pos + i);
        if (position_ok(p, W, H)) atomicAdd(pcnt + pixel_at(p.x, p.y, W), 1u);
    }
}

template <int CT>
__device__ __forceinline__ bool sample_ok(float4 p, typename ColorStore<CT>::T cr, float2 m, bool pok) {
    const float3 c = ColorStore<CT>::widen(cr);
    return pok && isfinite(c.x) && isfinite(c.y) && isfinite(c.z) && isfinite(m.x) && isfinite(m.y);
}

constexpr int kScatterWarps = 8;
constexpr int kScatterUnroll = 2;   // samples (and ticket atomics) in flight per thread

template <int CT>
__global__ void __launch_bounds__(32 * kScatterWarps) k_pix_scatter(
    const float4 *__restrict__ pos, const void *__restrict__ col, const float2 *__restrict__ mo,
    const float4 *__restrict__ world, uint32_t n, int W, int H, uint32_t *__restrict__ pcur, Bucket bk,
    uint32_t *__restrict__ accept, unsigned long long *__restrict__ dcount, DebugCheck dc) {
    using CS = ColorStore<CT>;
    __shared__ uint4 stage[kScatterWarps][32][5];   // 80-byte stride: conflict-free 16-byte accesses
    __shared__ uint32_t dest[kScatterWarps][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t step = gridDim.x * kScatterWarps * 32u * kScatterUnroll;
    for (uint32_t base = (blockIdx.x * kScatterWarps + w) * 32u * kScatterUnroll; base < n; base += step) {
        float4 p[kScatterUnroll];
        typename CS::T cr[kScatterUnroll];
        float2 m[kScatterUnroll];
#pragma unroll
        for (int r = 0; r < kScatterUnroll; ++r) {
            const uint32_t i = base + r * 32 + lane;
            p[r] = make_float4(-1.f, -1.f, 0.f, 0.f);
            if (i < n) {
                p[r] = __ldg(pos + i);
                cr[r] = CS::raw(col, i);
                m[r] = __ldg(mo + i);
            }
        }
        uint32_t d[kScatterUnroll];
        bool ok[kScatterUnroll];
#pragma unroll
        for (int r = 0; r < kScatterUnroll; ++r) {
            const uint32_t i = base + r * 32 + lane;
            const bool in = i < n;
            const bool pok = in && position_ok(p[r], W, H);
            ok[r] = in && sample_ok<CT>(p[r], cr[r], m[r], pok);
            agg_count(dcount + CNT_REJECTED, in && !ok[r]);
            if (in && accept) accept[i] = ok[r] ? 1u : 0u;
            d[r] = kInvalid;
            if (pok) {
                const uint32_t px = pixel_at(p[r].x, p[r].y, W);
                d[r] = atomicAdd(pcur + px, 1u);   // the cursors start at the bucket offsets
                if (!AFR_CHECK(d[r] < dc.cap, dc.derr)) d[r] = kInvalid;
            }
        }
#pragma unroll
        for (int r = 0; r < kScatterUnroll; ++r) {
            const uint32_t i = base + r * 32 + lane;
            if (d[r] != kInvalid) {
                float4 wp = make_float4(0.f, 0.f, 0.f, 0.f);
                if (ok[r] && world) wp = __ldg(world + i);
                uint4 q1;
                uint32_t my = 0u;
                if (CT == AFR_F32) {
                    const float4 cf = *reinterpret_cast<const float4 *>(&cr[r]);
                    q1 = make_uint4(__float_as_uint(cf.x), __float_as_uint(cf.y), __float_as_uint(cf.z),
                                    __float_as_uint(m[r].x));
                    my = __float_as_uint(m[r].y);
                } else {
                    const ushort4 h = *reinterpret_cast<const ushort4 *>(&cr[r]);
                    q1 = make_uint4((uint32_t)h.x | ((uint32_t)h.y << 16), (uint32_t)h.z, __float_as_uint(m[r].x),
                                    __float_as_uint(m[r].y));
                }
                stage[w][lane][0] = make_uint4(__float_as_uint(p[r].x), __float_as_uint(p[r].y),
                                               __float_as_uint(p[r].z), ok[r] ? i : kInvalid);
                stage[w][lane][1] = q1;
                stage[w][lane][2] = make_uint4(my, __float_as_uint(p[r].w), __float_as_uint(wp.x), __float_as_uint(wp.y));
                stage[w][lane][3] = make_uint4(__float_as_uint(wp.z), 0u, 0u, 0u);
            }
            dest[w][lane] = d[r];
            __syncwarp();
            // part u = 32 round + lane: part u % NP of record u / NP, so the NP
            // lanes of a record store its bytes contiguously
#pragma unroll
            for (int round = 0; round < NP; ++round) {
                const int u = round * 32 + lane, k = u / NP, q = u % NP;
                const uint32_t dk = dest[w][k];
                if (dk != kInvalid) bk.r[(size_t)NP * dk + q] = stage[w][k][q];
            }
            __syncwarp();
        }
    }
}

// ascending bitonic sort of one 64-bit key per lane across a full warp
__device__ __forceinline__ unsigned long long warp_sort_asc(unsigned long long v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, j);
            const bool up = ((lane & k) == 0), lower = ((lane & j) == 0);
            v = (lower == up) ? min(v, o) : max(v, o);
        }
    }
    return v;
}

// merge step of a bitonic sequence held across the warp into ascending order
__device__ __forceinline__ unsigned long long warp_merge_asc(unsigned long long v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int j = 16; j > 0; j >>= 1) {
        const unsigned long long o = __shfl_xor_sync(0xffffffffu, v, j);
        v = ((lane & j) == 0) ? min(v, o) : max(v, o);
    }
    return v;
}

// The 32 largest keys seen so far across the warp (ascending, lane 31 the
// largest) after one more key per lane (0: none; real keys are nonzero).
__device__ __forceinline__ unsigned long long warp_top32(unsigned long long top, unsigned long long key) {
    key = warp_sort_asc(key);
    const unsigned long long rev = __shfl_sync(0xffffffffu, key, 31 - (threadIdx.x & 31));
    return warp_merge_asc(max(top, rev));
}

// Queue state (count | head << 16) after m more pushes.
__device__ __forceinline__ uint32_t pushed_state(uint32_t st, uint32_t m, uint32_t ub) {
    const uint32_t cnt = st & 0xFFFFu, h = st >> 16;
    const uint32_t cn = (uint64_t)cnt + m < (uint64_t)ub ? cnt + m : ub;
    const uint32_t hn = (uint32_t)((h + (uint64_t)m) % ub);
    return cn | (hn << 16);
}

// Writes one kept record (parts a, q1, q2, q3) to queue slot dst.
template <int CT>
__device__ __forceinline__ void put_record(const uint4 &a, const uint4 &q1, const uint4 &q2, const uint4 &q3, size_t dst,
                                           uint32_t seq, const Queues &q) {
    q.xy[dst] = make_float2(__uint_as_float(a.x), __uint_as_float(a.y));
    q.t[dst] = __uint_as_float(a.z);
    q.depth[dst] = __uint_as_float(q2.y);
    q.seq[dst] = seq;
    if (CT == AFR_F32) {
        reinterpret_cast<float4 *>(q.col)[dst] =
            make_float4(__uint_as_float(q1.x), __uint_as_float(q1.y), __uint_as_float(q1.z), 0.f);
        q.mo[dst] = make_float2(__uint_as_float(q1.w), __uint_as_float(q2.x));
    } else {
        reinterpret_cast<ushort4 *>(q.col)[dst] =
            make_ushort4((unsigned short)(q1.x & 0xFFFFu), (unsigned short)(q1.x >> 16), (unsigned short)q1.y, 0);
        q.mo[dst] = make_float2(__uint_as_float(q1.z), __uint_as_float(q1.w));
    }
    if (q.world)
        q.world[dst] = make_float4(__uint_as_float(q2.z), __uint_as_float(q2.w), __uint_as_float(q3.x), 0.f);
}

// Thread per bucket record, pixels of up to kBigPixel records. A block takes
// kCommitTile consecutive records at a time and keeps their batch indices in
// shared memory, where the rank scans find all of a pixel's records but
// those of pixels crossing the tile's ends. state0 holds the queue states
// before the batch.
constexpr int kCommitTile = 256;

template <int CT>
__global__ void __launch_bounds__(kCommitTile) k_pix_commit(const uint32_t *__restrict__ poff, uint32_t P, int W,
                                                            int b, uint32_t seq0, Bucket bk, Queues q,
                                                            const uint32_t *__restrict__ state0, DebugCheck dc) {
    __shared__ uint32_t sidx[kCommitTile];
    uint32_t n = __ldg(poff + P);
    if (!AFR_CHECK(n <= dc.cap, dc.derr)) n = 0;
    const uint32_t ub = (uint32_t)b;
    const uint32_t *ridx = reinterpret_cast<const uint32_t *>(bk.r) + 3;   // batch index of record k: ridx[16 k]
    for (uint32_t t0 = blockIdx.x * (uint32_t)kCommitTile; t0 < n; t0 += gridDim.x * (uint32_t)kCommitTile) {
        const uint32_t e = t0 + threadIdx.x, t1 = min(t0 + (uint32_t)kCommitTile, n);
        uint4 a = make_uint4(0u, 0u, 0u, kInvalid), q1 = a, q2 = a, q3 = a;
        if (e < n) {
            a = __ldg(bk.r + (size_t)NP * e);
            q1 = __ldg(bk.r + (size_t)NP * e + 1);
            q2 = __ldg(bk.r + (size_t)NP * e + 2);
            if (q.world) q3 = __ldg(bk.r + (size_t)NP * e + 3);
        }
        sidx[threadIdx.x] = a.w;
        __syncthreads();
        // a record exists only for a valid position, so its pixel is in the image
        const uint32_t px = e < n ? pixel_at(__uint_as_float(a.x), __uint_as_float(a.y), W) : 0u;
        bool work = e < n && AFR_CHECK(px < P, dc.derr);
        uint32_t beg = 0, end = 0, st = 0;
        if (work) {
            beg = __ldg(poff + px);
            end = __ldg(poff + px + 1);
            st = __ldg(state0 + px);
            work = end - beg <= kBigPixel && (a.w != kInvalid || e == beg) && AFR_CHECK(end <= n, dc.derr);
        }
        if (work) {
            // batch indices are unique; a dead record's is kInvalid, above them all
            uint32_t rank = 0, dead = 0;
            const uint32_t s0 = max(beg, t0), s1 = min(end, t1);
            for (uint32_t k = beg; k < min(end, t0); ++k) {
                const uint32_t w = __ldg(ridx + (size_t)16 * k);
                rank += w < a.w;
                dead += w == kInvalid;
            }
            for (uint32_t k = s0; k < s1; ++k) {
                const uint32_t w = sidx[k - t0];
                rank += w < a.w;
                dead += w == kInvalid;
            }
            for (uint32_t k = max(beg, t1); k < end; ++k) {
                const uint32_t w = __ldg(ridx + (size_t)16 * k);
                rank += w < a.w;
                dead += w == kInvalid;
            }
            const uint32_t nl = end - beg - dead;
            if (e == beg) q.state[px] = pushed_state(st, nl, ub);
            if (a.w != kInvalid && rank + min(nl, ub) >= nl) {   // else evicted by newer samples of the batch
                const size_t dst = (size_t)px * ub + ((st >> 16) + rank) % ub;
                if (AFR_CHECK(dst < q.nslots, dc.derr)) put_record<CT>(a, q1, q2, q3, dst, seq0 + a.w, q);
            }
        }
        __syncthreads();   // the next tile overwrites sidx
    }
}

// Pixels of more than kBigPixel records: a warp streams the pixel's bucket,
// keeping the newest 32 live records by bitonic merges.
template <int CT>
__global__ void __launch_bounds__(256) k_pix_commit_big(const uint32_t *__restrict__ poff, uint32_t P, int b,
                                                        uint32_t seq0, Bucket bk, Queues q,
                                                        const uint32_t *__restrict__ state0, DebugCheck dc) {
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t ub = (uint32_t)b;
    const uint32_t *ridx = reinterpret_cast<const uint32_t *>(bk.r) + 3;
    const uint32_t n = __ldg(poff + P);
    for (uint32_t base = warp * 32u; base < P; base += nwarps * 32u) {
        const uint32_t p = base + (uint32_t)lane;
        uint32_t m = 0;
        if (p < P) m = __ldg(poff + p + 1) - __ldg(poff + p);
        unsigned big = __ballot_sync(0xffffffffu, m > kBigPixel);
        while (big) {
            const uint32_t px = base + (uint32_t)(__ffs(big) - 1);
            big &= big - 1u;
            const uint32_t beg = __ldg(poff + px);
            uint32_t end = __ldg(poff + px + 1);
            if (!AFR_CHECK(end <= n && n <= dc.cap, dc.derr)) end = beg;
            unsigned long long top = 0ull;
            uint32_t nl = 0;
            for (uint32_t k0 = beg; k0 < end; k0 += 32) {
                const uint32_t k = k0 + (uint32_t)lane;
                unsigned long long key = 0ull;
                if (k < end) {
                    const uint32_t w = __ldg(ridx + (size_t)16 * k);
                    if (w != kInvalid) key = ((unsigned long long)(w + 1u) << 32) | k;
                }
                nl += (uint32_t)__popc(__ballot_sync(0xffffffffu, key != 0ull));
                top = warp_top32(top, key);
            }
            const uint32_t st = __ldg(state0 + px);
            if (lane == 0) q.state[px] = pushed_state(st, nl, ub);
            const uint32_t kept = min(nl, ub);
            if (lane >= 32 - (int)kept) {
                const uint32_t k = (uint32_t)top, rank = nl - 32u + (uint32_t)lane;   // position in insertion order
                const size_t dst = (size_t)px * ub + ((st >> 16) + rank) % ub;
                if (AFR_CHECK(dst < q.nslots && k < end, dc.derr)) {
                    const uint4 a = __ldg(bk.r + (size_t)NP * k);
                    const uint4 q1 = __ldg(bk.r + (size_t)NP * k + 1);
                    const uint4 q2 = __ldg(bk.r + (size_t)NP * k + 2);
                    uint4 q3 = make_uint4(0u, 0u, 0u, 0u);
                    if (q.world) q3 = __ldg(bk.r + (size_t)NP * k + 3);
                    put_record<CT>(a, q1, q2, q3, dst, seq0 + a.w, q);
                }
            }
        }
    }
}

template <int CT>
cudaError_t run(AfrContext *c, const float4 *pos, const void *col, const float2 *mo, const float4 *world, uint32_t n,
                uint32_t seq0, cudaStream_t s, cudaEvent_t queues_free, bool reset) {
    const uint32_t P = (uint32_t)c->P;
    const DebugCheck dc{(uint32_t)c->batch_cap, c->derr};
    Bucket bk{c->bucket};
    cudaError_t e;
    // binning: the context's scratch only (the scatter counts the rejected samples)
    if (reset && (e = cudaMemsetAsync(c->dcount + CNT_REJECTED, 0, sizeof(unsigned long long), s)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(c->ccnt, 0, sizeof(uint32_t) * P, s)) != cudaSuccess) return e;
    k_pix_count<<<grid_for(n, 256), 256, 0, s>>>(pos, n, c->W, c->H, c->ccnt);
    if ((e = scan_exclusive(c->ccnt, c->coff, P, c->scan_tmp_in, s)) != cudaSuccess) return e;
    // append cursors start at the bucket offsets: a ticket is the record's place
    if ((e = cudaMemcpyAsync(c->ccur, c->coff, sizeof(uint32_t) * P, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return e;
    const int gs = grid_for((n + kScatterUnroll - 1) / kScatterUnroll, 32 * kScatterWarps);
    uint32_t *accept = c->fifo_n ? c->fifo_flag : nullptr;
    k_pix_scatter<CT><<<gs, 32 * kScatterWarps, 0, s>>>(pos, col, mo, c->r_world ? world : nullptr, n, c->W, c->H,
                                                        c->ccur, bk, accept, c->dcount, dc);
    // from here on the queues: wait until they are free, clear them if asked
    if (queues_free && (e = cudaStreamWaitEvent(s, queues_free, 0)) != cudaSuccess) return e;
    if (reset) {
        static_assert(CNT_REJECTED == 0, "the rejected count comes first");
        if ((e = cudaMemsetAsync(c->r_state, 0, sizeof(uint32_t) * P, s)) != cudaSuccess) return e;
        if ((e = cudaMemsetAsync(c->dcount + 1, 0, sizeof(unsigned long long) * (CNT_N - 1), s)) != cudaSuccess)
            return e;
        if (c->q_total && (e = cudaMemsetAsync(c->q_total, 0, sizeof(uint32_t), s)) != cudaSuccess) return e;
    }
    // the cursors are spent: they take the queue states before the batch,
    // which every commit thread reads
    if ((e = cudaMemcpyAsync(c->ccur, c->r_state, sizeof(uint32_t) * P, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return e;
    Queues q{c->r_xy, c->r_mo, c->r_t, c->r_depth, c->r_seq, c->r_col, c->r_state, c->r_world, c->nslots};
    k_pix_commit<CT><<<grid_for(n, kCommitTile), kCommitTile, 0, s>>>(c->coff, P, c->W, c->b, seq0, bk, q, c->ccur,
                                                                      dc);
    k_pix_commit_big<CT><<<grid_for(P, 256), 256, 0, s>>>(c->coff, P, c->b, seq0, bk, q, c->ccur, dc);
    return cudaGetLastError();
}

}  // namespace

namespace {

// ---- reconstructor queue (section 5.2) ----------------------------------------
// The batch's accepted samples (the scatter flagged them) enter the
// N-slot queue in index order: a scan gives each its rank r among the
// batch's accepted samples, and it lands at slot (total + r) mod N; of a batch
// with more than N accepted samples only the last N are written.
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

cudaError_t launch_ingest(AfrContext *c, const AfrSampleBatch *batch, uint32_t n, uint32_t seq0,
                          cudaStream_t s, cudaEvent_t queues_free, bool reset) {
    const float4 *pos = reinterpret_cast<const float4 *>(batch->pos_dev);
    const float2 *mo = reinterpret_cast<const float2 *>(batch->motion_dev);
    const void *col = batch->color_dev;
    const float4 *world = reinterpret_cast<const float4 *>(batch->world_dev);
    switch (c->ct) {
        case AFR_F32: return run<AFR_F32>(c, pos, col, mo, world, n, seq0, s, queues_free, reset);
        case AFR_F16: return run<AFR_F16>(c, pos, col, mo, world, n, seq0, s, queues_free, reset);
        default: return run<AFR_BF16>(c, pos, col, mo, world, n, seq0, s, queues_free, reset);
    }
}

}  // namespace afr

// k_ingest.cu -- section 4 deep buffer: push a batch of samples into the
// per-pixel queues of depth b (each keeps its b newest samples by insertion
// order).
//
// The batch arrives in insertion order with its samples spread over the whole
// image, and the queues are planes in pixel order, so ingest is a sort. It
// runs through cells of 16 x 8 pixels:
//
//  1. count:   per bucket, the samples whose position is valid (reads only
//              the 16-byte position of each sample). A cell's records go to
//              kSubBuckets buckets by batch index modulo kSubBuckets, laid out
//              one after another, so that the cell's bucket is still one
//              contiguous range while each counter takes one eighth of the
//              cell's atomics.
//  2. scan:    bucket offsets.
//  3. scatter: each sample appends its 64-byte record (position, colour,
//              motion, batch index, hit point) to its bucket. A warp stages its
//              32 records in shared memory and stores each with four lanes, so
//              every store is two whole sectors; a thread takes the tickets of
//              several samples before using any, to keep atomics in flight. A
//              sample whose colour or motion is not finite leaves a dead
//              record (batch index kInvalid).
//  4. commit:  one CTA per cell reads its bucket once, sorts the records by
//              pixel in shared memory, ranks each pixel's records by batch
//              index (insertion order) and writes the newest min(b, m) to the
//              queue slots (head + rank) mod b that sequential pushes would
//              use, so a warp's stores cover consecutive slots. A cell with
//              more records than one round of shared memory is committed in
//              rounds over groups of its pixels; a pixel that alone holds
//              more is ranked by a warp streaming the bucket and keeping the
//              newest 32 in registers.
#include "afr_internal.cuh"

namespace afr {
namespace {

constexpr int kCellW = 16, kCellH = 8, kCellPix = kCellW * kCellH;
constexpr int kSubBuckets = 8;
constexpr int kCommitCap = 3072;      // records of one round in shared memory
constexpr int kCommitThreads = 512;
constexpr int kCommitWarps = kCommitThreads / 32;

// Bucket records, NP = 4 uint4 (64 bytes: two whole sectors) each:
//   q0 = (x, y, t, batch index)
//   q1 = FP32: (r, g, b, m_x); 16-bit: (r | g << 16, b, m_x, m_y)
//   q2 = (m_y for FP32 colours, depth, hit point X, Y)
//   q3 = (hit point Z, 0, 0, 0)
// The first 16 bytes are all the commit's sort reads. (Three-part, 48-byte
// records, whose halves of a shared sector L2 has to merge, measured slower.)
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

__device__ __forceinline__ uint32_t cell_of(float x, float y, int ncx) {
    const int qx = (int)floorf(x), qy = (int)floorf(y);
    return (uint32_t)((qy / kCellH) * ncx + qx / kCellW);
}

__global__ void __launch_bounds__(256) k_cell_count(const float4 *__restrict__ pos, uint32_t n, int W, int H, int ncx,
                                                    uint32_t *__restrict__ ccnt) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 p = __ldg(pos + i);
        if (position_ok(p, W, H)) atomicAdd(ccnt + cell_of(p.x, p.y, ncx) * kSubBuckets + (i & (kSubBuckets - 1)), 1u);
    }
}

template <int CT>
__device__ __forceinline__ bool sample_ok(float4 p, typename ColorStore<CT>::T cr, float2 m, bool pok) {
    const float3 c = ColorStore<CT>::widen(cr);
    return pok && isfinite(c.x) && isfinite(c.y) && isfinite(c.z) && isfinite(m.x) && isfinite(m.y);
}

constexpr int kScatterWarps = 8;
constexpr int kScatterUnroll = 4;   // samples (and ticket atomics) in flight per thread

template <int CT, int NP>
__global__ void __launch_bounds__(32 * kScatterWarps) k_cell_scatter(
    const float4 *__restrict__ pos, const void *__restrict__ col, const float2 *__restrict__ mo,
    const float4 *__restrict__ world, uint32_t n, int W, int H, int ncx, const uint32_t *__restrict__ coff,
    uint32_t *__restrict__ ccur, Bucket bk, uint32_t *__restrict__ accept, unsigned long long *__restrict__ dcount,
    DebugCheck dc) {
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
                const uint32_t key = cell_of(p[r].x, p[r].y, ncx) * kSubBuckets + (i & (kSubBuckets - 1));
                d[r] = __ldg(coff + key) + atomicAdd(ccur + key, 1u);
                if (!AFR_CHECK(d[r] < dc.cap, dc.derr)) d[r] = kInvalid;
            }
        }
#pragma unroll
        for (int r = 0; r < kScatterUnroll; ++r) {
            const uint32_t i = base + r * 32 + lane;
            if (d[r] != kInvalid) {
                float4 wp = make_float4(0.f, 0.f, 0.f, 0.f);
                if (NP == 4 && ok[r] && world) wp = __ldg(world + i);
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
                if (NP == 4) stage[w][lane][3] = make_uint4(__float_as_uint(wp.z), 0u, 0u, 0u);
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

// Shared memory of the commit kernel (dynamic; kCommitCap records a round).
struct CommitSmem {
    uint32_t *idx;      // [cap] batch index of round record k
    uint32_t *src;      // [cap] its bucket position within the cell
    uint16_t *tick;     // [cap] its arrival rank within its pixel in this round
    uint8_t *lp;        // [cap] its cell pixel
    uint32_t *sidx;     // [cap] batch indices in pixel order (sorted position u)
    uint32_t *ssrc;     // [cap] bucket positions in pixel order
    uint8_t *slp;       // [cap] cell pixels in pixel order
    uint32_t *total;    // [kCellPix] the batch's records per pixel
    uint32_t *count;    // [kCellPix] this round's records per pixel
    uint32_t *start;    // [kCellPix] first sorted position of each pixel in this round
    uint32_t *state;    // [kCellPix] queue state of each pixel before the batch
    uint32_t *misc;     // [2] records gathered in this round, end of this round's pixels
};

constexpr size_t kCommitSmemBytes =
    (size_t)kCommitCap * (4 + 4 + 2 + 1 + 4 + 4 + 1) + (size_t)kCellPix * 16 + 16;

__device__ __forceinline__ CommitSmem commit_smem(unsigned char *base) {
    CommitSmem m;
    unsigned char *p = base;
    auto take = [&](size_t bytes) {
        unsigned char *r = p;
        p += (bytes + 15) & ~(size_t)15;
        return r;
    };
    m.idx = reinterpret_cast<uint32_t *>(take(4 * kCommitCap));
    m.src = reinterpret_cast<uint32_t *>(take(4 * kCommitCap));
    m.sidx = reinterpret_cast<uint32_t *>(take(4 * kCommitCap));
    m.ssrc = reinterpret_cast<uint32_t *>(take(4 * kCommitCap));
    m.total = reinterpret_cast<uint32_t *>(take(4 * kCellPix));
    m.count = reinterpret_cast<uint32_t *>(take(4 * kCellPix));
    m.start = reinterpret_cast<uint32_t *>(take(4 * kCellPix));
    m.state = reinterpret_cast<uint32_t *>(take(4 * kCellPix));
    m.misc = reinterpret_cast<uint32_t *>(take(16));
    m.tick = reinterpret_cast<uint16_t *>(take(2 * kCommitCap));
    m.lp = reinterpret_cast<uint8_t *>(take(kCommitCap));
    m.slp = reinterpret_cast<uint8_t *>(take(kCommitCap));
    return m;
}

constexpr int kCommitUnroll = 4;   // bucket records in flight per thread (gather)
constexpr int kPutUnroll = 2;      // kept records in flight per thread (queue writes)

// Writes kept records (bucket position src, queue slot dst, sequence number)
// field by field, the loads of each field issued together.
template <int CT, int NP>
__device__ __forceinline__ void put_entries(const Bucket &bk, uint32_t c0, uint32_t (&src)[kPutUnroll],
                                            const size_t (&dst)[kPutUnroll], const uint32_t (&seq)[kPutUnroll],
                                            const Queues &q, const DebugCheck &dc) {
#pragma unroll
    for (int r = 0; r < kPutUnroll; ++r)   // dc.cap: bucket records; q.nslots: queue slots
        if (src[r] != kInvalid && !AFR_CHECK(c0 + src[r] < dc.cap && dst[r] < q.nslots, dc.derr)) src[r] = kInvalid;
    uint4 a[kPutUnroll], q2[kPutUnroll];
#pragma unroll
    for (int r = 0; r < kPutUnroll; ++r)
        if (src[r] != kInvalid) {
            a[r] = bk.r[(size_t)NP * (c0 + src[r])];
            q2[r] = bk.r[(size_t)NP * (c0 + src[r]) + 2];
        }
#pragma unroll
    for (int r = 0; r < kPutUnroll; ++r)
        if (src[r] != kInvalid) {
            q.xy[dst[r]] = make_float2(__uint_as_float(a[r].x), __uint_as_float(a[r].y));
            q.t[dst[r]] = __uint_as_float(a[r].z);
            q.depth[dst[r]] = __uint_as_float(q2[r].y);
            q.seq[dst[r]] = seq[r];
        }
    uint4 bb[kPutUnroll];
#pragma unroll
    for (int r = 0; r < kPutUnroll; ++r)
        if (src[r] != kInvalid) bb[r] = bk.r[(size_t)NP * (c0 + src[r]) + 1];
#pragma unroll
    for (int r = 0; r < kPutUnroll; ++r)
        if (src[r] != kInvalid) {
            if (CT == AFR_F32) {
                reinterpret_cast<float4 *>(q.col)[dst[r]] =
                    make_float4(__uint_as_float(bb[r].x), __uint_as_float(bb[r].y), __uint_as_float(bb[r].z), 0.f);
                q.mo[dst[r]] = make_float2(__uint_as_float(bb[r].w), __uint_as_float(q2[r].x));
            } else {
                reinterpret_cast<ushort4 *>(q.col)[dst[r]] =
                    make_ushort4((unsigned short)(bb[r].x & 0xFFFFu), (unsigned short)(bb[r].x >> 16),
                                 (unsigned short)bb[r].y, 0);
                q.mo[dst[r]] = make_float2(__uint_as_float(bb[r].z), __uint_as_float(bb[r].w));
            }
            if (NP == 4 && q.world) {
                const uint4 q3 = bk.r[(size_t)NP * (c0 + src[r]) + 3];
                q.world[dst[r]] = make_float4(__uint_as_float(q2[r].z), __uint_as_float(q2[r].w),
                                              __uint_as_float(q3.x), 0.f);
            }
        }
}

template <int CT, int NP>
__global__ void __launch_bounds__(kCommitThreads, 2) k_cell_commit(const uint32_t *__restrict__ coff, int W, int H,
                                                                   int ncx, int b, uint32_t seq0, Bucket bk, Queues q,
                                                                   DebugCheck dc) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const CommitSmem sm = commit_smem(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t cell = blockIdx.x;
    const uint32_t c0 = coff[cell * kSubBuckets], nc = coff[(cell + 1) * kSubBuckets] - c0;
    if (nc == 0) return;   // block-uniform
    const int x0 = (int)(cell % (uint32_t)ncx) * kCellW, y0 = (int)(cell / (uint32_t)ncx) * kCellH;
    const uint32_t ub = (uint32_t)b;
    // image pixel of cell pixel l (inside the image for every l that holds a record)
    auto pixel_of = [&](uint32_t l) -> size_t {
        return (size_t)(y0 + (int)(l / kCellW)) * (size_t)W + (size_t)(x0 + (int)(l % kCellW));
    };
    // cell pixel of a bucket record, kCellPix for a dead record
    auto local_of = [&](uint32_t i, uint4 a) -> uint32_t {
        if (i == kInvalid) return kCellPix;
        return (uint32_t)(((int)floorf(__uint_as_float(a.y)) - y0) * kCellW + ((int)floorf(__uint_as_float(a.x)) - x0));
    };
    const bool multi = nc > (uint32_t)kCommitCap;
    for (int l = tid; l < kCellPix; l += kCommitThreads) {
        const int x = x0 + l % kCellW, y = y0 + l / kCellW;
        sm.state[l] = (x < W && y < H) ? q.state[(size_t)y * W + x] : 0u;
        sm.total[l] = 0;
    }
    __syncthreads();
    if (multi) {
        // per-pixel totals, to group the pixels into rounds
        for (uint32_t j = tid; j < nc; j += kCommitThreads) {
            const uint4 a = bk.r[(size_t)NP * (c0 + j)];
            const uint32_t l = local_of(a.w, a);
            if (l < kCellPix) atomicAdd(&sm.total[l], 1u);
        }
        __syncthreads();
        // a pixel alone above one round: a warp streams the bucket
        for (int l = warp; l < kCellPix; l += kCommitWarps) {
            const uint32_t m = sm.total[l];
            if (m <= (uint32_t)kCommitCap) continue;
            unsigned long long top = 0ull;
            for (uint32_t base = 0; base < nc; base += 32) {
                const uint32_t j = base + (uint32_t)lane;
                unsigned long long key = 0ull;
                if (j < nc) {
                    const uint4 a = bk.r[(size_t)NP * (c0 + j)];
                    if (local_of(a.w, a) == (uint32_t)l) key = ((unsigned long long)(a.w + 1u) << 32) | j;
                }
                top = warp_top32(top, key);
            }
            const uint32_t kept = min(m, ub);
            uint32_t src[kPutUnroll], seq[kPutUnroll];
#pragma unroll
            for (int r = 0; r < kPutUnroll; ++r) src[r] = kInvalid;
            size_t dst[kPutUnroll];
            if (lane >= 32 - (int)kept) {
                const uint32_t rank = m - 32u + (uint32_t)lane;   // position in insertion order
                src[0] = (uint32_t)top;
                seq[0] = seq0 + (uint32_t)(top >> 32) - 1u;
                dst[0] = pixel_of(l) * ub + ((sm.state[l] >> 16) + rank) % ub;
            }
            put_entries<CT, NP>(bk, c0, src, dst, seq, q, dc);
        }
    }
    uint32_t group_begin = 0;
    while (group_begin < (uint32_t)kCellPix) {
        if (tid == 0) {
            uint32_t e = kCellPix;
            if (multi) {
                uint32_t acc = 0;
                for (e = group_begin; e < (uint32_t)kCellPix; ++e) {
                    const uint32_t m = sm.total[e];
                    if (m > (uint32_t)kCommitCap) continue;   // streamed above
                    if (acc + m > (uint32_t)kCommitCap) break;
                    acc += m;
                }
            }
            sm.misc[1] = e;
            sm.misc[0] = 0;
        }
        for (int l = tid; l < kCellPix; l += kCommitThreads) sm.count[l] = 0;
        __syncthreads();
        const uint32_t ge = sm.misc[1];
        // gather the round's records, kCommitUnroll bucket loads in flight per
        // thread; a single round keeps record j at place j (dead ones unused)
        for (uint32_t base = 0; base < nc; base += kCommitThreads * kCommitUnroll) {
            uint32_t ii[kCommitUnroll];
            uint4 aa[kCommitUnroll];
#pragma unroll
            for (int r = 0; r < kCommitUnroll; ++r) {
                const uint32_t j = base + tid + r * kCommitThreads;
                ii[r] = kInvalid;
                if (j < nc) {
                    aa[r] = bk.r[(size_t)NP * (c0 + j)];
                    ii[r] = aa[r].w;
                }
            }
#pragma unroll
            for (int r = 0; r < kCommitUnroll; ++r) {
                const uint32_t j = base + tid + r * kCommitThreads;
                const uint32_t l = local_of(ii[r], aa[r]);
                // a single round marks every place: src[j] == j for a record
                // gathered at j, kInvalid for a dead record (shared memory
                // holds earlier blocks' values otherwise)
                if (!multi && j < nc && l == kCellPix) sm.src[j] = kInvalid;
                if (l < group_begin || l >= ge || (multi && sm.total[l] > (uint32_t)kCommitCap)) continue;
                const uint32_t k = multi ? atomicAdd(&sm.misc[0], 1u) : j;
                sm.idx[k] = ii[r];
                sm.src[k] = j;
                sm.lp[k] = (uint8_t)l;
                sm.tick[k] = (uint16_t)atomicAdd(&sm.count[l], 1u);
            }
        }
        __syncthreads();
        if (warp == 0) {   // exclusive scan of the counts (128 = 4 per lane)
            uint32_t v[4], sum = 0;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                v[r] = sm.count[lane * 4 + r];
                sum += v[r];
            }
            uint32_t incl = sum;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            uint32_t run = incl - sum;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                sm.start[lane * 4 + r] = run;
                run += v[r];
            }
            if (lane == 31) sm.misc[0] = run;   // the round's records
        }
        if (!multi)
            for (int l = tid; l < kCellPix; l += kCommitThreads) sm.total[l] = sm.count[l];
        __syncthreads();
        const uint32_t nr = sm.misc[0];
        // copies of the round's records in pixel order
        if (multi) {
            for (uint32_t k = tid; k < nr; k += kCommitThreads) {
                const uint32_t l = sm.lp[k], u = sm.start[l] + sm.tick[k];
                sm.sidx[u] = sm.idx[k];
                sm.ssrc[u] = sm.src[k];
                sm.slp[u] = (uint8_t)l;
            }
        } else {
            for (uint32_t j = tid; j < nc; j += kCommitThreads) {
                if (sm.src[j] != j) continue;   // a dead record's place
                const uint32_t l = sm.lp[j], u = sm.start[l] + sm.tick[j];
                sm.sidx[u] = sm.idx[j];
                sm.ssrc[u] = j;
                sm.slp[u] = (uint8_t)l;
            }
        }
        __syncthreads();
        // up to 32 records in a pixel: a thread per record counts the pixel's
        // records with a smaller batch index (batch indices are unique)
        for (uint32_t u0 = 0; u0 < nr; u0 += kCommitThreads * kPutUnroll) {
            uint32_t src[kPutUnroll], seq[kPutUnroll];
            size_t dst[kPutUnroll];
#pragma unroll
            for (int r = 0; r < kPutUnroll; ++r) {
                const uint32_t u = u0 + tid + r * kCommitThreads;
                src[r] = kInvalid;
                if (u >= nr) continue;
                const uint32_t l = sm.slp[u], m = sm.count[l];
                if (m > 32u) continue;
                const uint32_t beg = sm.start[l], me = sm.sidx[u];
                uint32_t rank = 0;
                for (uint32_t v = beg; v < beg + m; ++v) rank += sm.sidx[v] < me;
                if (rank + min(m, ub) < m) continue;   // evicted by newer samples of the batch
                src[r] = sm.ssrc[u];
                seq[r] = seq0 + me;
                dst[r] = pixel_of(l) * ub + ((sm.state[l] >> 16) + rank) % ub;
            }
            put_entries<CT, NP>(bk, c0, src, dst, seq, q, dc);
        }
        // more than 32: a warp keeps the newest 32 by bitonic merges of the
        // pixel's records, 32 at a time
        for (uint32_t l = group_begin + (uint32_t)warp; l < ge; l += kCommitWarps) {
            const uint32_t m = sm.count[l];
            if (m <= 32u) continue;
            const uint32_t beg = sm.start[l];
            unsigned long long top = 0ull;
            for (uint32_t base = 0; base < m; base += 32) {
                unsigned long long key = 0ull;
                if (base + (uint32_t)lane < m) {
                    const uint32_t u = beg + base + lane;
                    key = ((unsigned long long)(sm.sidx[u] + 1u) << 32) | u;
                }
                top = warp_top32(top, key);
            }
            const uint32_t kept = min(m, ub);
            uint32_t src[kPutUnroll], seq[kPutUnroll];
#pragma unroll
            for (int r = 0; r < kPutUnroll; ++r) src[r] = kInvalid;
            size_t dst[kPutUnroll];
            if (lane >= 32 - (int)kept) {
                const uint32_t u = (uint32_t)top, rank = m - 32u + (uint32_t)lane;
                src[0] = sm.ssrc[u];
                seq[0] = seq0 + sm.sidx[u];
                dst[0] = pixel_of(l) * ub + ((sm.state[l] >> 16) + rank) % ub;
            }
            put_entries<CT, NP>(bk, c0, src, dst, seq, q, dc);
        }
        __syncthreads();
        group_begin = ge;
    }
    // queue states after pushing each pixel's records
    for (int l = tid; l < kCellPix; l += kCommitThreads) {
        const uint32_t m = sm.total[l];
        if (m == 0) continue;
        const uint32_t st = sm.state[l], cnt = st & 0xFFFFu, h = st >> 16;
        const uint32_t cn = (uint64_t)cnt + m < (uint64_t)ub ? cnt + m : ub;
        const uint32_t hn = (uint32_t)((h + (uint64_t)m) % ub);
        q.state[pixel_of((uint32_t)l)] = cn | (hn << 16);
    }
}

template <int CT>
cudaError_t run(AfrContext *c, const float4 *pos, const void *col, const float2 *mo, const float4 *world, uint32_t n,
                uint32_t seq0, cudaStream_t s) {
    const int ncx = (c->W + kCellW - 1) / kCellW;
    const int nkeys = c->ncells * kSubBuckets;
    const DebugCheck dc{(uint32_t)c->batch_cap, c->derr};
    Bucket bk{c->bucket};
    static bool attr_set = false;   // per colour type: raise the commit kernels' shared-memory limit once
    cudaError_t e = cudaSuccess;
    if (!attr_set) {
        e = cudaFuncSetAttribute(k_cell_commit<CT, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kCommitSmemBytes);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if ((e = cudaMemsetAsync(c->ccnt, 0, sizeof(uint32_t) * nkeys, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->ccur, 0, sizeof(uint32_t) * nkeys, s)) != cudaSuccess) return e;
    const int g = grid_for(n, 256);
    k_cell_count<<<g, 256, 0, s>>>(pos, n, c->W, c->H, ncx, c->ccnt);
    if ((e = scan_exclusive(c->ccnt, c->coff, nkeys, c->scan_tmp, s)) != cudaSuccess) return e;
    const int gs = grid_for((n + kScatterUnroll - 1) / kScatterUnroll, 32 * kScatterWarps);
    uint32_t *accept = c->fifo_n ? c->fifo_flag : nullptr;
    Queues q{c->r_xy, c->r_mo, c->r_t, c->r_depth, c->r_seq, c->r_col, c->r_state, c->r_world, c->nslots};
    k_cell_scatter<CT, 4><<<gs, 32 * kScatterWarps, 0, s>>>(pos, col, mo, c->r_world ? world : nullptr, n, c->W, c->H,
                                                             ncx, c->coff, c->ccur, bk, accept, c->dcount, dc);
    k_cell_commit<CT, 4><<<c->ncells, kCommitThreads, kCommitSmemBytes, s>>>(c->coff, c->W, c->H, ncx, c->b, seq0, bk,
                                                                             q, dc);
    return cudaGetLastError();
}

}  // namespace

int ingest_sub_buckets() { return kSubBuckets; }

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

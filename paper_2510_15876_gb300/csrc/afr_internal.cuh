// afr_internal.cuh -- context layout and device helpers shared by the CUDA
// translation units of the reconstruction library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string>

#include "../../include/afr.h"

namespace afr {

constexpr uint32_t kInvalid = 0xFFFFFFFFu;
constexpr int kMaxDepth = 32;
constexpr float kAgeDecay = 3.47f;               // section 4: exp(-3.47 a)
constexpr float kLumR = 0.2126f, kLumG = 0.7152f, kLumB = 0.0722f;  // Rec. 709
constexpr float kSigmaSMin = 0.5f, kSigmaTMin = 0.05f;
constexpr float kLog2e = 1.4426950408889634f;
constexpr int kSortedBinMax = 4096;              // frame bins ordered by seq up to this size

// device counters (unsigned long long)
enum { CNT_REJECTED = 0, CNT_DROPPED, CNT_UNSORTED, CNT_RESIDENT, CNT_BIG, CNT_N };
// device status word bits
enum { ERR_TIMEOUT = 1u, ERR_CHECK = 2u };

// Device-side consistency checks (builds with AFR_DEBUG): a failed check sets
// ERR_CHECK in the context's status word, which afr_get_status reports, and
// the caller skips the access it guarded. Release builds compile the checks
// out (AFR_CHECK is the constant true and its condition is not evaluated).
#ifdef AFR_DEBUG
__device__ __forceinline__ bool dcheck(bool ok, uint32_t *derr) {
    if (!ok) atomicOr(derr, (uint32_t)ERR_CHECK);
    return ok;
}
#define AFR_CHECK(cond, derr) ::afr::dcheck((cond), (derr))
#else
#define AFR_CHECK(cond, derr) true
#endif

// Bounds of one array for the checks: its element count and the status word.
struct DebugCheck {
    uint32_t cap;
    uint32_t *derr;
};

// Per-tile partial statistics written by the gradient pass (64 bytes). The
// luminance moments are FP64 because a tile above 4096 samples merges its
// warps' moments in FP64; everything else is an integer count or an FP32 sum.
struct alignas(16) TilePartial {
    double sw;         // sum of age weights
    double mean;       // weighted mean luminance
    double m2;         // weighted sum of squared deviations
    float sgx, sgy, sgt;   // gradient sums over non-empty pixels
    uint32_t n;        // samples
    uint32_t nonempty; // non-empty pixels
    uint32_t pad[3];
};
static_assert(sizeof(TilePartial) == 64, "one 64-byte record per tile");

// Rows 0, 1 and 3 of a row-major view-projection matrix (camera reprojection).
struct Camera {
    float m[12];
};

// Per-context record of a batched launch (device memory).
struct BatchCtx {
    int W, H, R, S, ntx, tbx, th, ntiles_x;
    float window, eps;
    AfrParams prm;
    const float4 *grad;
    const TilePartial *tiles;
    float2 *sigma;
    float4 *fconst;
    const uint32_t *amin2;
    const uint32_t *foff;
    const float4 *fpos;
    const void *fcol;
    float4 *out;
    uint32_t *derr;
    uint32_t fcap;      // frame-view record capacity (checks)
    uint32_t a0;        // first work item (tile) of this context
    uint32_t s0;        // first width chunk of this context
};

}  // namespace afr

struct AfrContext {
    AfrConfig cfg{};
    int W = 0, H = 0, b = 0, S = 0, R = 0, ct = 0;
    int P = 0;
    int ntx = 0, nty = 0, ntiles = 0;
    size_t nslots = 0;        // P * b
    int csize = 16;           // bytes per stored colour (16 for F32, 8 for 16-bit)

    // deep buffer, slot index p*b + s (storage order, circular per pixel)
    float2 *r_xy = nullptr;
    float2 *r_mo = nullptr;
    float *r_t = nullptr;
    float *r_depth = nullptr;
    uint32_t *r_seq = nullptr;
    void *r_col = nullptr;
    uint32_t *r_state = nullptr;  // count | head << 16

    // ingest scratch
    // reconstructor queue of section 5.2 (fifo_capacity > 0): slot k of N
    size_t fifo_n = 0;
    float2 *q_xy = nullptr, *q_mo = nullptr;
    float *q_t = nullptr;
    uint32_t *q_seq = nullptr;
    void *q_col = nullptr;
    uint32_t *q_total = nullptr;  // [1] accepted samples so far (the next slot is q_total mod N)
    float4 *q_world = nullptr;    // [N] hit points (world_points contexts)
    float4 *r_world = nullptr;    // [P*b] hit point of each queue slot (world_points contexts)
    uint32_t *fifo_flag = nullptr;  // [batch_cap] 1 for an accepted sample
    uint32_t *fifo_rank = nullptr;  // [batch_cap + 1] exclusive scan of fifo_flag, then the total
    uint32_t *fifo_scan = nullptr;  // scan block sums for batch_cap entries
    // ingest scratch: per-cell counts and offsets (cells of 16 x 8 pixels) and
    // the batch's records bucketed by pixel (batch_cap records)
    uint32_t *ccnt = nullptr;     // [P] bucket counts
    uint32_t *coff = nullptr;     // [P + 1] bucket offsets
    uint32_t *ccur = nullptr;     // [P] append cursors, then the queue states before the batch
    uint4 *bucket = nullptr;      // [4 * batch_cap] 64-byte sample records in bucket order
    size_t batch_cap = 0;

    // maps
    float2 *lbar = nullptr;       // [P] weighted mean luminance as double-float (hi, lo)
    float4 *grad = nullptr;       // [P] (Gx, Gy, Gt, Lbar)
    float4 *pstat = nullptr;      // [P] (sum w, mean L, M2, Gt)
    float2 *sigma = nullptr;      // [P] (sigma_s, sigma_t)
    double *tile_terms = nullptr;   // [8 ntiles] per-tile terms of afr_tile_error (64 B a tile)
    float4 *fconst = nullptr;     // [P] gather constants (-ks, -kt, exponent shift m, disc radius as int bits)
    float *cov_r[2] = {nullptr, nullptr};   // [P] footprint radii of adaptive reconstructions (ping-pong)
    int32_t *cov_n = nullptr;     // [P] samples in each pixel's footprint in the last adaptive reconstruction
    int cov_cur = 0;              // cov_r[cov_cur] holds the radii of the last adaptive reconstruction
    bool cov_init = false;        // the coverage state holds its start values
    bool adaptive_last = false;   // the last reconstruction used adaptive footprints
    uint32_t *amin2 = nullptr;    // [P] float bits of min a^2 per frame bin
    afr::TilePartial *tiles = nullptr;  // [ntiles]

    // frame view
    uint32_t *fcnt = nullptr;     // [P]
    uint32_t *foff = nullptr;     // [P+1]
    float4 *fpos = nullptr;       // [frame_cap] (x', y', a^2, bin column as int bits)
    void *fcol = nullptr;         // [frame_cap]
    uint32_t *fseq = nullptr;     // [frame_cap] sequence numbers
    uint32_t *flist = nullptr;    // [frame_cap] each bin's source slots, unordered (reprojection scratch)
    uint32_t *flseq = nullptr;    // [frame_cap] their sequence numbers
    size_t frame_cap = 0;

    // scan scratch
    uint32_t *scan_tmp = nullptr;       // scan block sums of the reprojection
    uint32_t *scan_tmp_in = nullptr;    // ... of the ingest (it may run beside the reprojection)
    size_t scan_tmp_n = 0;

    // backward scratch
    float4 *bgrad = nullptr;      // [P] per-pixel (g_r/S, g_g/S, g_b/S, valid)
    float *bparam = nullptr;      // [n_bblocks * 6] per-block parameter-gradient partials
    int n_bblocks = 0;

    unsigned long long *dcount = nullptr;  // [CNT_N]
    uint32_t *derr = nullptr;

    // host-side state
    uint64_t inserted = 0;
    bool grads_valid = false;
    float grads_t = 0.f;
    bool frame_valid = false;
    float frame_t = 0.f;
    bool recon_valid = false;
    float recon_t = 0.f;
    AfrParams recon_params{};
    bool sigma_imported = false;
    int tile_bx = 4;              // filter CTA tile: (2*tile_bx) x (64/tile_bx) pixels (8 x 16 measured fastest at 1080p16)
    // filter kernel timing (afr_profile_filter): event pairs, launches recorded
    cudaEvent_t *prof_ev = nullptr;
    bool prof_on = false, prof_capture_hit = false;
    int prof_n = 0;
    std::string err;
};

namespace afr {

// ---- colour storage ----------------------------------------------------------
template <int CT> struct ColorStore;
template <> struct ColorStore<AFR_F32> {
    using T = float4;
    static __device__ __forceinline__ float3 load(const void *base, size_t i) {
        float4 v = __ldg(reinterpret_cast<const float4 *>(base) + i);
        return make_float3(v.x, v.y, v.z);
    }
    static __device__ __forceinline__ T raw(const void *base, size_t i) {
        return __ldg(reinterpret_cast<const float4 *>(base) + i);
    }
    static __device__ __forceinline__ float3 widen(T v) { return make_float3(v.x, v.y, v.z); }
};
template <> struct ColorStore<AFR_F16> {
    using T = ushort4;
    static __device__ __forceinline__ float3 widen(T v) {
        return make_float3(__half2float(__ushort_as_half(v.x)), __half2float(__ushort_as_half(v.y)),
                           __half2float(__ushort_as_half(v.z)));
    }
    static __device__ __forceinline__ T raw(const void *base, size_t i) {
        return __ldg(reinterpret_cast<const ushort4 *>(base) + i);
    }
    static __device__ __forceinline__ float3 load(const void *base, size_t i) { return widen(raw(base, i)); }
};
template <> struct ColorStore<AFR_BF16> {
    using T = ushort4;
    static __device__ __forceinline__ float bf(unsigned short h) {
        return __uint_as_float(((unsigned)h) << 16);
    }
    static __device__ __forceinline__ float3 widen(T v) { return make_float3(bf(v.x), bf(v.y), bf(v.z)); }
    static __device__ __forceinline__ T raw(const void *base, size_t i) {
        return __ldg(reinterpret_cast<const ushort4 *>(base) + i);
    }
    static __device__ __forceinline__ float3 load(const void *base, size_t i) { return widen(raw(base, i)); }
};

__device__ __forceinline__ float luminance(float3 c) {
    return fmaf(kLumB, c.z, fmaf(kLumG, c.y, kLumR * c.x));
}

// ---- double-float arithmetic ------------------------------------------------
// A value held as the unevaluated sum h + l of two floats (|l| <= ulp(h)/2),
// about 48 significant bits from FP32 operations only. Built on the error-free
// transformations TwoSum (Knuth) and TwoProduct with a fused multiply-add
// (Ogita, Rump and Oishi, "Accurate sum and dot product", 2005). The spatial
// and temporal gradients subtract luminances that agree in most of their
// bits; holding the luminances and their weighted means in this form keeps
// those differences accurate to FP32 rounding of the difference itself.
struct dfloat {
    float h, l;
};

__device__ __forceinline__ dfloat two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ dfloat fast_two_sum(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfloat two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
    const dfloat s = two_sum(a.h, b.h);
    const dfloat t = two_sum(a.l, b.l);
    dfloat r = fast_two_sum(s.h, __fadd_rn(s.l, t.h));
    return fast_two_sum(r.h, __fadd_rn(r.l, t.l));
}
__device__ __forceinline__ dfloat df_mul(dfloat a, float b) {
    dfloat p = two_prod(a.h, b);
    return fast_two_sum(p.h, __fmaf_rn(a.l, b, p.l));
}
__device__ __forceinline__ dfloat df_div(dfloat a, dfloat b) {
    const float q1 = __fdiv_rn(a.h, b.h);
    const dfloat r = df_add(a, df_mul({-b.h, -b.l}, q1));
    const float q2 = __fdiv_rn(r.h, b.h);
    return fast_two_sum(q1, q2);
}
// a - b rounded once to float
__device__ __forceinline__ float df_diff(dfloat a, dfloat b) {
    return __fadd_rn(__fsub_rn(a.h, b.h), __fsub_rn(a.l, b.l));
}

// Rec. 709 luminance in double-float: each weight is split into the float
// nearest to it and the float nearest to the remainder.
__device__ __forceinline__ dfloat luminance_df(float3 c) {
    constexpr double kR = 0.2126, kG = 0.7152, kB = 0.0722;
    constexpr float rh = (float)kR, gh = (float)kG, bh = (float)kB;
    constexpr float rl = (float)(kR - (double)rh), gl = (float)(kG - (double)gh), bl = (float)(kB - (double)bh);
    dfloat s = df_mul({rh, rl}, c.x);
    s = df_add(s, df_mul({gh, gl}, c.y));
    return df_add(s, df_mul({bh, bl}, c.z));
}

// 2^x with the hardware approximation (relative error below 2^-22).
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Rounds of key grouping before the remaining lanes fall back to one atomic
// each: each round takes the lowest pending lane's key and ballots the lanes
// that share it (a shuffle and a ballot, far cheaper here than a
// __match_any_sync); samples moving together give a warp a few distinct keys,
// while keys spread at random are left to per-lane atomics after the rounds.
constexpr int kGroupRounds = 4;

// Warp-aggregated atomic add of 1 at base[key]: lanes with equal keys share
// one atomic (up to kGroupRounds keys a warp); returns this lane's ticket.
// Tickets of one key are distinct and dense; their order is unspecified.
__device__ __forceinline__ uint32_t agg_inc(uint32_t *base, uint32_t key) {
    const unsigned active = __activemask();
    const int lane = threadIdx.x & 31;
    unsigned todo = active, mine = 0u;
    int my_leader = lane;
    uint32_t first = 0;
    for (int round = 0; round < kGroupRounds && todo; ++round) {
        const int leader = __ffs(todo) - 1;
        const uint32_t k = __shfl_sync(active, key, leader);
        const unsigned peers = __ballot_sync(active, key == k);
        if (lane == leader) first = atomicAdd(base + k, (uint32_t)__popc(peers));
        if (key == k) {
            mine = peers;
            my_leader = leader;
        }
        todo &= ~peers;
    }
    if (todo & (1u << lane)) return atomicAdd(base + key, 1u);
    return __shfl_sync(active & ~todo, first, my_leader) + __popc(mine & ((1u << lane) - 1u));
}

// Warp-aggregated count of lanes with flag set, added to *ctr.
__device__ __forceinline__ void agg_count(unsigned long long *ctr, bool flag) {
    unsigned mask = __activemask();
    unsigned bits = __ballot_sync(mask, flag);
    if ((threadIdx.x & 31) == __ffs(mask) - 1 && bits) atomicAdd(ctr, (unsigned long long)__popc(bits));
}

// Multiprocessor count of the current device (read once per device).
int device_sms();

// Blocks for n items of a grid-stride kernel: at most 32 blocks per SM.
inline int grid_for(size_t n, int block, int cap = 0) {
    if (cap <= 0) cap = 32 * device_sms();
    size_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > (size_t)cap) g = cap;
    return (int)g;
}

// ---- launch wrappers (one per translation unit) ------------------------------
// Each returns cudaSuccess or the launch error.
cudaError_t scan_exclusive(const uint32_t *in, uint32_t *out, size_t n, uint32_t *tmp, cudaStream_t s);
size_t scan_tmp_elems(size_t n);

// queues_free: the steps that touch the queues wait for it (may be null);
// reset: the queues, the reconstructor queue and the counters are cleared
// before the commit (the rejected count at the start).
cudaError_t launch_ingest(AfrContext *c, const AfrSampleBatch *batch, uint32_t n, uint32_t seq0,
                          cudaStream_t s, cudaEvent_t queues_free = nullptr, bool reset = false);
cudaError_t launch_fifo_append(AfrContext *c, const AfrSampleBatch *batch, uint32_t n, uint32_t seq0, cudaStream_t s);
cudaError_t launch_gradients(AfrContext *c, float t_now, cudaStream_t s);
cudaError_t launch_reproject(AfrContext *c, float t_now, const Camera *cam, cudaStream_t s);
cudaError_t launch_sigma(AfrContext *c, const AfrParams *prm, bool keep, bool adaptive, cudaStream_t s);
cudaError_t launch_coverage_init(AfrContext *c, cudaStream_t s);
cudaError_t launch_filter(AfrContext *c, float t_now, bool adaptive, float4 *out, cudaStream_t s);
cudaError_t launch_feedback(AfrContext *c, AfrTileStats *out, cudaStream_t s);
cudaError_t launch_tile_error(AfrContext *c, float kappa, float lambda, float importance, const uint32_t *occluded,
                              float *E, AfrGain *gain, cudaStream_t s);
cudaError_t launch_backward(AfrContext *c, const float4 *grad_rgb, float *grad_col, float *grad_prm,
                            cudaStream_t s);
cudaError_t launch_set_frame_colors(AfrContext *c, const float *rgb, cudaStream_t s);
int backward_blocks(int W, int H);
cudaError_t launch_batch(int ct, const BatchCtx *cs, int nctx, uint32_t nchunks, uint32_t total, uint32_t *queue,
                         int grid, cudaStream_t s);
constexpr int kBatchSigmaChunk = 2048;   // pixels per width chunk of a batched launch
constexpr int kBatchDirectPixels = 131072;   // larger contexts of a batch get their own launches
constexpr int kBatchWorkers = 4;             // streams of afr_batch_refresh
cudaError_t launch_resident_count(AfrContext *c, cudaStream_t s);

}  // namespace afr

// k_reproject.cu -- section 6.2: move every buffered sample to the display
// time along its screen velocity and rebin it into the frame view (a CSR
// over destination pixels), ordered within each bin by sequence number.
//
//  count:  thread per queue slot; x' = x + m_x (t_now - t) with one rounding
//          per operation (__fmul_rn / __fadd_rn, so no contraction), drops
//          samples leaving the image and counts per destination bin (the
//          lanes of a warp grouped by bin with one match instruction).
//  scan:   bin offsets.
//  list:   each moved sample (its bin kept by the count pass, 4 bytes a
//          slot) writes its slot index and its sequence number into its bin's
//          lists (unordered, 8 bytes a sample), at the ticket its bin's cursor
//          returns (the cursors start at the bin offsets).
//  place:  thread per frame record, in bin order: the slot of list entry e
//          is moved again, its rank in the bin is the number of sequence
//          numbers in the bin's list below its own (sequence numbers are
//          unique), and it writes (x', y', a^2, bin column), its colour and its
//          sequence number to the bin's offset + rank. The lanes of a warp
//          mostly share a bin, so the rank scans are broadcast reads and the
//          record writes cover whole sectors; the frame view, and every sum
//          over it, is deterministic without a reorder pass over the records.
//          Each bin's smallest a^2 (the filter's exponent shift) is the
//          minimum over the bin's warp segments, one atomic each.
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

// Section 6.2 with camera matrices: the stored hit point rendered by the
// current camera, plus the sample's own screen motion times its age; each
// matrix row summed left to right, one rounding per operation.
__device__ __forceinline__ float cam_row(const Camera &c, int r, float4 w) {
    float v = __fmul_rn(c.m[4 * r], w.x);
    v = __fadd_rn(v, __fmul_rn(c.m[4 * r + 1], w.y));
    v = __fadd_rn(v, __fmul_rn(c.m[4 * r + 2], w.z));
    return __fadd_rn(v, c.m[4 * r + 3]);
}

__device__ __forceinline__ Moved move_camera(float4 w, float2 m, float t, float t_now, int W, int H,
                                             const Camera &cam) {
    Moved r;
    const float cx = cam_row(cam, 0, w), cy = cam_row(cam, 1, w), cw = cam_row(cam, 2, w);
    const float sx = __fmul_rn(__fadd_rn(__fmul_rn(__fdiv_rn(cx, cw), 0.5f), 0.5f), (float)W);
    const float sy = __fmul_rn(__fadd_rn(__fmul_rn(__fdiv_rn(cy, cw), 0.5f), 0.5f), (float)H);
    const float a = __fsub_rn(t_now, t);
    r.xp = __fadd_rn(sx, __fmul_rn(m.x, a));
    r.yp = __fadd_rn(sy, __fmul_rn(m.y, a));
    r.a2 = __fmul_rn(a, a);
    r.ok = cw > 0.f && r.xp >= 0.f && r.xp < (float)W && r.yp >= 0.f && r.yp < (float)H;
    r.bin = r.ok ? (uint32_t)(int)floorf(r.yp) * (uint32_t)W + (uint32_t)(int)floorf(r.xp) : kInvalid;
    return r;
}

// slot i -> (pixel, storage slot); b is a power of two in the common case
__device__ __forceinline__ void split_slot(uint32_t i, int b, int bshift, uint32_t &p, int &s) {
    if (bshift >= 0) {
        p = i >> bshift;
        s = (int)(i & (uint32_t)(b - 1));
    } else {
        p = i / (uint32_t)b;
        s = (int)(i - p * (uint32_t)b);
    }
}

__device__ __forceinline__ bool slot_live(uint32_t st, int s, int b) {
    int n = (int)(st & 0xFFFFu), h = (int)(st >> 16);
    int age = h - 1 - s;
    if (age < 0) age += b;
    return age < n;
}

// FIFO: the slots are the reconstructor queue's, live below min(*state, nslots)
// (state then points at its count of accepted samples). The slot's data is
// loaded together with its pixel's state (one round trip, not two).
template <bool FIFO, bool CAM>
__device__ __forceinline__ bool live_move(uint32_t i, uint32_t nlive, int b, int bshift, int W, int H, float t_now,
                                          const Camera &cam, const float4 *__restrict__ world,
                                          const uint32_t *__restrict__ state, const float2 *__restrict__ r_xy,
                                          const float2 *__restrict__ r_mo, const float *__restrict__ r_t, Moved &mv,
                                          bool &live) {
    uint32_t p = 0, st = 0;
    int s = 0;
    live = false;
    if (FIFO) {
        if (i >= nlive) return false;
    } else {
        split_slot(i, b, bshift, p, s);
        st = __ldg(state + p);
    }
    float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
    float2 xy = make_float2(0.f, 0.f);
    if (CAM) w = __ldg(world + i);
    else xy = __ldg(r_xy + i);
    const float2 m = __ldg(r_mo + i);
    const float t = __ldg(r_t + i);
    if (!FIFO && !slot_live(st, s, b)) return false;
    live = true;
    mv = CAM ? move_camera(w, m, t, t_now, W, H, cam) : move_sample(xy, m, t, t_now, W, H);
    return mv.ok;
}

// A warp takes kCountRows rows of 32 slots at a time, their loads issued
// together.
constexpr int kCountRows = 4;
template <bool FIFO, bool CAM>
__global__ void __launch_bounds__(256) k_count(uint32_t nslots, int b, int bshift, int W, int H, float t_now,
                                               Camera cam, const float4 *__restrict__ world,
                                               const uint32_t *__restrict__ state, const float2 *__restrict__ r_xy,
                                               const float2 *__restrict__ r_mo, const float *__restrict__ r_t,
                                               uint32_t *__restrict__ fcnt, uint32_t *__restrict__ sbin,
                                               unsigned long long *__restrict__ dcount) {
    const uint32_t nlive = FIFO ? min(__ldg(state), nslots) : 0u;
    const int lane = threadIdx.x & 31;
    uint32_t dropped = 0;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i0 = warp * 32u * kCountRows; i0 < nslots; i0 += nwarps * 32u * kCountRows) {
        Moved mv[kCountRows];
        bool live[kCountRows];
#pragma unroll
        for (int r = 0; r < kCountRows; ++r) {
            const uint32_t i = i0 + (uint32_t)(r * 32 + lane);
            mv[r].ok = false;
            live[r] = false;
            if (i < nslots)
                live_move<FIFO, CAM>(i, nlive, b, bshift, W, H, t_now, cam, world, state, r_xy, r_mo, r_t, mv[r],
                                     live[r]);
        }
#pragma unroll
        for (int r = 0; r < kCountRows; ++r) {
            const uint32_t i = i0 + (uint32_t)(r * 32 + lane);
            dropped += live[r] && !mv[r].ok;
            const uint32_t key = mv[r].ok ? mv[r].bin : kInvalid;
            if (i < nslots) sbin[i] = key;
            const unsigned peers = __match_any_sync(0xffffffffu, key);
            if (mv[r].ok && lane == __ffs(peers) - 1) atomicAdd(fcnt + mv[r].bin, (uint32_t)__popc(peers));
        }
    }
    const uint32_t d = __reduce_add_sync(0xffffffffu, dropped);
    if (lane == 0 && d) atomicAdd(dcount + CNT_DROPPED, (unsigned long long)d);
}

// The slots' bins from the count pass (kInvalid: dead or moved out). A warp
// takes kListRows rows of 32 slots at a time and issues every row's ticket
// atomic before it reads any back, so the atomics' latencies overlap.
constexpr int kListRows = 8;
__global__ void __launch_bounds__(256) k_list(uint32_t nslots, const uint32_t *__restrict__ sbin,
                                              const uint32_t *__restrict__ r_seq, uint32_t *__restrict__ fcur, uint32_t *__restrict__ flist,
                                              uint32_t *__restrict__ flseq, DebugCheck dc) {
    const int lane = threadIdx.x & 31;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i0 = warp * 32u * kListRows; i0 < nslots; i0 += nwarps * 32u * kListRows) {
        uint32_t bin[kListRows], sq[kListRows], first[kListRows];
        unsigned peers[kListRows];
#pragma unroll
        for (int r = 0; r < kListRows; ++r) {
            const uint32_t i = i0 + (uint32_t)(r * 32 + lane);
            bin[r] = kInvalid;
            sq[r] = 0;
            if (i < nslots) {
                bin[r] = __ldg(sbin + i);
                sq[r] = __ldg(r_seq + i);
            }
        }
#pragma unroll
        for (int r = 0; r < kListRows; ++r) {
            peers[r] = __match_any_sync(0xffffffffu, bin[r]);
            first[r] = 0;
            if (bin[r] != kInvalid && lane == __ffs(peers[r]) - 1)
                first[r] = atomicAdd(fcur + bin[r], (uint32_t)__popc(peers[r]));
        }
#pragma unroll
        for (int r = 0; r < kListRows; ++r) {
            const uint32_t i = i0 + (uint32_t)(r * 32 + lane);
            const uint32_t f = __shfl_sync(0xffffffffu, first[r], bin[r] != kInvalid ? __ffs(peers[r]) - 1 : lane);
            if (bin[r] == kInvalid) continue;
            const uint32_t at = f + __popc(peers[r] & ((1u << lane) - 1u));
            if (AFR_CHECK(at < dc.cap, dc.derr)) {
                flist[at] = i;
                flseq[at] = sq[r];
            }
        }
    }
}

// fcnt holds every bin's end here (the list's cursors); a bin above
// kSortedBinMax records takes its ranks by counting it down (arrival order)
// and is counted as unsorted.
// The frame records arrive in bin order, so the lanes of a warp that share a
// bin are one segment: its smallest a^2 goes to amin2 with one atomic (the
// filter's exponent shift; bit order = value order for a^2 >= 0).
template <int CT, bool FIFO, bool CAM>
__global__ void __launch_bounds__(256) k_place(int W, int H, float t_now, Camera cam, const float4 *__restrict__ world,
                                               const float2 *__restrict__ r_xy, const float2 *__restrict__ r_mo,
                                               const float *__restrict__ r_t, const uint32_t *__restrict__ r_seq,
                                               const void *__restrict__ r_col, uint32_t P,
                                               const uint32_t *__restrict__ foff, const uint32_t *__restrict__ flist,
                                               const uint32_t *__restrict__ flseq, uint32_t *__restrict__ fcnt,
                                               uint32_t *__restrict__ amin2, float4 *__restrict__ fpos,
                                               void *__restrict__ fcol, uint32_t *__restrict__ fseq,
                                               unsigned long long *__restrict__ dcount, DebugCheck dc, uint32_t nsrc) {
    using CS = ColorStore<CT>;
    uint32_t n = __ldg(foff + P);
    if (!AFR_CHECK(n <= dc.cap, dc.derr)) n = 0;
    const int lane = threadIdx.x & 31;
    const uint32_t stride = gridDim.x * blockDim.x;
    // warp-uniform trip count: every lane of a warp reaches the match below
    for (uint32_t e0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); e0 < n; e0 += stride) {
        const uint32_t e = e0 + (uint32_t)lane;
        uint32_t i = 0;
        bool ok = e < n;
        if (ok) {
            i = __ldg(flist + e);
            ok = AFR_CHECK(i < nsrc, dc.derr);
        }
        Moved mv;
        mv.ok = false;
        mv.bin = kInvalid;
        if (ok)
            mv = CAM ? move_camera(__ldg(world + i), __ldg(r_mo + i), __ldg(r_t + i), t_now, W, H, cam)
                     : move_sample(__ldg(r_xy + i), __ldg(r_mo + i), __ldg(r_t + i), t_now, W, H);
        const uint32_t key = mv.ok ? mv.bin : kInvalid;
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        if (!mv.ok) continue;
        const uint32_t bits = __reduce_min_sync(peers, __float_as_uint(mv.a2));
        if (lane == __ffs(peers) - 1) atomicMin(amin2 + mv.bin, bits);
        const uint32_t sq = __ldg(flseq + e);
        const uint32_t beg = __ldg(foff + mv.bin), end = __ldg(foff + mv.bin + 1);
        uint32_t rank = 0;
        if (end - beg <= (uint32_t)kSortedBinMax) {
            for (uint32_t k = beg; k < end; ++k) rank += __ldg(flseq + k) < sq;
        } else {
            rank = atomicSub(fcnt + mv.bin, 1u) - 1u - beg;   // the cursor ends at the bin's end
            if (rank == 0) atomicAdd(dcount + CNT_UNSORTED, 1ull);
        }
        const uint32_t d = beg + rank;
        if (!AFR_CHECK(d < n, dc.derr)) continue;
        fpos[d] = make_float4(mv.xp, mv.yp, mv.a2, __int_as_float((int)floorf(mv.xp)));
        reinterpret_cast<typename CS::T *>(fcol)[d] = CS::raw(r_col, i);
        fseq[d] = sq;
    }
}

__global__ void k_fill_u32(uint32_t *p, size_t n, uint32_t v) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

}  // namespace

cudaError_t launch_reproject(AfrContext *c, float t_now, const Camera *camp, cudaStream_t s) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(c->fcnt, 0, sizeof(uint32_t) * c->P, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c->dcount + CNT_DROPPED, 0, sizeof(unsigned long long) * 2, s)) != cudaSuccess) return e;
    k_fill_u32<<<grid_for(c->P, 256), 256, 0, s>>>(c->amin2, c->P, 0x7f800000u);
    // source: the per-pixel queues, or the reconstructor queue (section 5.2);
    // moved by screen motion, or rendered by a camera (hit points)
    const bool fifo = c->fifo_n > 0, cam = camp != nullptr;
    const Camera cm = cam ? *camp : Camera{};
    const size_t nsrc = fifo ? c->fifo_n : c->nslots;
    const uint32_t *state = fifo ? c->q_total : c->r_state;
    const float2 *xy = fifo ? c->q_xy : c->r_xy, *mo = fifo ? c->q_mo : c->r_mo;
    const float *tt = fifo ? c->q_t : c->r_t;
    const uint32_t *sq = fifo ? c->q_seq : c->r_seq;
    const void *col = fifo ? c->q_col : c->r_col;
    const float4 *wp = fifo ? c->q_world : c->r_world;
    const int g = grid_for(nsrc, 256);
    const uint32_t ns = (uint32_t)nsrc;
    const int bshift = (c->b & (c->b - 1)) == 0 ? __builtin_ctz((unsigned)c->b) : -1;
    const DebugCheck dc{(uint32_t)c->frame_cap, c->derr};
#define AFR_COUNT(F_, C_)                                                                                    \
    k_count<F_, C_><<<g, 256, 0, s>>>(ns, c->b, bshift, c->W, c->H, t_now, cm, wp, state, xy, mo, tt, c->fcnt, \
                                      c->fseq, c->dcount)
    if (fifo && cam) AFR_COUNT(true, true);
    else if (fifo) AFR_COUNT(true, false);
    else if (cam) AFR_COUNT(false, true);
    else AFR_COUNT(false, false);
#undef AFR_COUNT
    if ((e = scan_exclusive(c->fcnt, c->foff, c->P, c->scan_tmp, s)) != cudaSuccess) return e;
    // the list's append cursors start at the bin offsets (a ticket is the entry's place)
    if ((e = cudaMemcpyAsync(c->fcnt, c->foff, sizeof(uint32_t) * c->P, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
        return e;
    // fseq holds each slot's bin until the placement pass writes the frame
    k_list<<<g, 256, 0, s>>>(ns, c->fseq, sq, c->fcnt, c->flist, c->flseq, dc);
#define AFR_PLACE(CT_, F_, C_)                                                                                     \
    k_place<CT_, F_, C_><<<g, 256, 0, s>>>(c->W, c->H, t_now, cm, wp, xy, mo, tt, sq, col, (uint32_t)c->P, c->foff, \
                                           c->flist, c->flseq, c->fcnt, c->amin2, c->fpos, c->fcol, c->fseq,       \
                                           c->dcount, dc, ns)
#define AFR_REPROJ(CT_)                                                                                        \
    do {                                                                                                       \
        if (fifo && cam) AFR_PLACE(CT_, true, true);                                                           \
        else if (fifo) AFR_PLACE(CT_, true, false);                                                            \
        else if (cam) AFR_PLACE(CT_, false, true);                                                             \
        else AFR_PLACE(CT_, false, false);                                                                     \
    } while (0)
    switch (c->ct) {
        case AFR_F32: AFR_REPROJ(AFR_F32); break;
        case AFR_F16: AFR_REPROJ(AFR_F16); break;
        default: AFR_REPROJ(AFR_BF16); break;
    }
#undef AFR_REPROJ
#undef AFR_PLACE
    return cudaGetLastError();
}

}  // namespace afr

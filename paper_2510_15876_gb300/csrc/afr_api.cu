// afr_api.cu -- the C ABI of include/afr.h: context life cycle, argument and
// call-order checks, and the stream-ordered launch sequence of each call.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "afr_internal.cuh"
#ifdef AFR_DEBUG
#include "../../include/afr_debug.h"
#endif

using afr::grid_for;

namespace {

// One NVTX range per ABI call (free when no profiler is attached).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

#ifdef AFR_DEBUG
// Allocation-failure injection (afr_debug_fail_alloc): the device allocation
// with this index and every later one fail as if the device were full.
int g_fail_after = -1;
int g_allocs = 0;
#endif

// Every device allocation of the library goes through here.
cudaError_t dmalloc(void **p, size_t bytes) {
    *p = nullptr;
#ifdef AFR_DEBUG
    if (g_fail_after >= 0 && g_allocs++ >= g_fail_after) return cudaErrorMemoryAllocation;
#endif
    return cudaMalloc(p, bytes ? bytes : 1);
}

AfrStatus fail(AfrContext *c, AfrStatus st, const char *msg) {
    if (c) c->err = msg;
    return st;
}

AfrStatus cuda_fail(AfrContext *c, cudaError_t e, const char *where) {
    if (c) {
        c->err = std::string(where) + ": " + cudaGetErrorString(e);
    }
    return e == cudaErrorMemoryAllocation ? AFR_ERR_OOM : AFR_ERR_CUDA;
}

template <typename T>
cudaError_t dalloc(T **p, size_t n) {
    return dmalloc(reinterpret_cast<void **>(p), (n ? n : 1) * sizeof(T));
}

void free_all(AfrContext *c) {
    void *ptrs[] = {c->r_xy, c->r_mo, c->r_t, c->r_depth, c->r_seq, c->r_col, c->r_state, c->bucket, c->fifo_flag, c->fifo_rank, c->fifo_scan,
                    c->ccnt, c->coff, c->ccur, c->lbar, c->grad, c->pstat, c->sigma, c->tile_terms, c->fconst, c->cov_r[0], c->cov_r[1], c->cov_n, c->amin2, c->tiles, c->fcnt,
                    c->foff, c->fpos, c->fcol, c->fseq, c->flist, c->flseq, c->q_xy, c->q_mo, c->q_t, c->q_seq, c->q_col, c->q_total, c->q_world, c->r_world, c->scan_tmp, c->scan_tmp_in, c->bgrad, c->bparam, c->dcount, c->derr};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

bool aligned(const void *p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// IEEE binary16 bits to float, from the format's definition.
float half_to_float(uint16_t h) {
    int sgn = (h >> 15) & 1, ex = (h >> 10) & 31, man = h & 1023;
    float v;
    if (ex == 0) v = std::ldexp((float)man, -24);
    else if (ex == 31) v = man ? NAN : INFINITY;
    else v = std::ldexp((float)(man + 1024), ex - 25);
    return sgn ? -v : v;
}

float bf16_to_float(uint16_t h) {
    uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

void widen_colors(int ct, const void *src, size_t i, float *dst3) {
    if (ct == AFR_F32) {
        const float *f = static_cast<const float *>(src) + 4 * i;
        dst3[0] = f[0]; dst3[1] = f[1]; dst3[2] = f[2];
    } else {
        const uint16_t *h = static_cast<const uint16_t *>(src) + 4 * i;
        for (int k = 0; k < 3; ++k) dst3[k] = ct == AFR_F16 ? half_to_float(h[k]) : bf16_to_float(h[k]);
    }
}

}  // namespace

namespace afr {

int device_sms() {
    constexpr int kMaxDevices = 64;
    static int cached[kMaxDevices] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return 1;
    }
    if (cached[dev] == 0) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
            cudaGetLastError();
            return 1;
        }
        cached[dev] = sms;
    }
    return cached[dev];
}

namespace {
__global__ void k_resident(const uint32_t *state, int P, unsigned long long *out) {
    unsigned long long acc = 0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) acc += state[p] & 0xFFFFu;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc) atomicAdd(out, acc);
}
}  // namespace
cudaError_t launch_resident_count(AfrContext *c, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(c->dcount + CNT_RESIDENT, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    k_resident<<<grid_for(c->P, 256), 256, 0, s>>>(c->r_state, c->P, c->dcount + CNT_RESIDENT);
    return cudaGetLastError();
}
}  // namespace afr

struct AfrBatch {
    std::vector<AfrContext *> ctxs;  // queue order (largest first)
    std::vector<int> user_index;     // caller's index of each queue position
    std::vector<int> tile_bx;        // tile shape each context had at creation
    afr::BatchCtx *h_ctx = nullptr;  // pinned staging of the device records
    afr::BatchCtx *d_ctx = nullptr;
    uint32_t *d_queue = nullptr;
    int n_direct = 0;                // leading contexts (largest) reconstructed by direct launches
    uint32_t total = 0;              // work items of the persistent kernel (tiles of the other contexts)
    uint32_t nchunks = 0;            // width chunks of the other contexts
    int ct = 0, grid = 0;
    // afr_batch_refresh: worker streams forked from and joined to the caller's
    // stream, and each context's worker (longest-processing-time first)
    std::vector<cudaStream_t> workers;
    std::vector<cudaEvent_t> joined;
    cudaEvent_t forked = nullptr;
    std::vector<int> worker_of;      // per queue position
};

extern "C" {

AfrStatus afr_create(const AfrConfig *cfg, AfrContext **out) {
    Range nvtx_range("afr_create");
    if (!cfg || !out) return AFR_ERR_INVALID_ARG;
    *out = nullptr;
    const AfrConfig &g = *cfg;
    if (g.width < 1 || g.height < 1 || g.width > 16384 || g.height > 16384 || g.depth < 1 ||
        g.depth > afr::kMaxDepth || g.tile < 1 || g.tile > 256 || g.radius < 0 || g.radius > 8 ||
        g.color_type < AFR_F32 || g.color_type > AFR_BF16 || !(g.window > 0.f) || !std::isfinite(g.window) ||
        !(g.eps_grad > 0.f) || !(g.undersample_m >= 0.f))
        return AFR_ERR_INVALID_ARG;
    if ((size_t)g.width * g.height * g.depth > (1ull << 28)) return AFR_ERR_INVALID_ARG;
    if (g.fifo_capacity > (1u << 28)) return AFR_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return AFR_ERR_CUDA;
    }
    AfrContext *c = new (std::nothrow) AfrContext();
    if (!c) return AFR_ERR_OOM;
    c->cfg = g;
    c->W = g.width;
    c->H = g.height;
    c->b = g.depth;
    c->S = g.tile;
    c->R = g.radius;
    c->ct = g.color_type;
    c->P = c->W * c->H;
    c->ntx = (c->W + c->S - 1) / c->S;
    c->nty = (c->H + c->S - 1) / c->S;
    c->ntiles = c->ntx * c->nty;
    c->nslots = (size_t)c->P * c->b;
    c->csize = c->ct == AFR_F32 ? 16 : 8;
    c->fifo_n = g.fifo_capacity;
    c->frame_cap = std::max(c->nslots, c->fifo_n);
    c->scan_tmp_n = afr::scan_tmp_elems((size_t)c->P);
    c->n_bblocks = afr::backward_blocks(c->W, c->H);
    cudaError_t e = cudaSuccess;
    size_t P = c->P, N = c->nslots;
#define AFR_ALLOC(ptr, n)                           \
    if (e == cudaSuccess) e = dalloc(&(ptr), (n));
    AFR_ALLOC(c->r_xy, N);
    AFR_ALLOC(c->r_mo, N);
    AFR_ALLOC(c->r_t, N);
    AFR_ALLOC(c->r_depth, N);
    AFR_ALLOC(c->r_seq, N);
    if (e == cudaSuccess) e = dmalloc(&c->r_col, N * c->csize);
    AFR_ALLOC(c->r_state, P);
    const size_t nkeys = P;   // ingest buckets: one per pixel
    AFR_ALLOC(c->ccnt, nkeys);
    AFR_ALLOC(c->coff, nkeys + 1);
    AFR_ALLOC(c->ccur, nkeys);
    AFR_ALLOC(c->lbar, P);
    AFR_ALLOC(c->grad, P);
    AFR_ALLOC(c->pstat, P);
    AFR_ALLOC(c->sigma, P);
    AFR_ALLOC(c->fconst, P);
    AFR_ALLOC(c->tile_terms, (size_t)8 * c->ntiles);
    AFR_ALLOC(c->cov_r[0], P);
    AFR_ALLOC(c->cov_r[1], P);
    AFR_ALLOC(c->cov_n, P);
    AFR_ALLOC(c->amin2, P);
    AFR_ALLOC(c->tiles, (size_t)c->ntiles);
    AFR_ALLOC(c->fcnt, P);
    AFR_ALLOC(c->foff, P + 1);
    if (g.world_points) AFR_ALLOC(c->r_world, N);
    if (c->fifo_n) {
        const size_t Q = c->fifo_n;
        if (g.world_points) AFR_ALLOC(c->q_world, Q);
        AFR_ALLOC(c->q_xy, Q);
        AFR_ALLOC(c->q_mo, Q);
        AFR_ALLOC(c->q_t, Q);
        AFR_ALLOC(c->q_seq, Q);
        if (e == cudaSuccess) e = dmalloc(&c->q_col, Q * c->csize);
        AFR_ALLOC(c->q_total, 1);
        if (e == cudaSuccess) e = cudaMemset(c->q_total, 0, sizeof(uint32_t));
    }
    AFR_ALLOC(c->fpos, c->frame_cap);
    if (e == cudaSuccess) e = dmalloc(&c->fcol, c->frame_cap * c->csize);
    AFR_ALLOC(c->fseq, c->frame_cap);
    AFR_ALLOC(c->flist, c->frame_cap);
    AFR_ALLOC(c->flseq, c->frame_cap);
    AFR_ALLOC(c->scan_tmp, c->scan_tmp_n);
    AFR_ALLOC(c->scan_tmp_in, c->scan_tmp_n);
    AFR_ALLOC(c->bgrad, 2 * P);
    AFR_ALLOC(c->bparam, (size_t)c->n_bblocks * 6);
    AFR_ALLOC(c->dcount, (size_t)afr::CNT_N);
    AFR_ALLOC(c->derr, 1);
#undef AFR_ALLOC
    if (e == cudaSuccess) e = cudaMemset(c->r_state, 0, P * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(c->foff, 0, (P + 1) * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemset(c->dcount, 0, afr::CNT_N * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(c->derr, 0, sizeof(uint32_t));
    if (e == cudaSuccess) e = afr::launch_coverage_init(c, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        AfrStatus st = e == cudaErrorMemoryAllocation ? AFR_ERR_OOM : AFR_ERR_CUDA;
        cudaGetLastError();
        free_all(c);
        delete c;
        return st;
    }
    *out = c;
    return AFR_OK;
}

void afr_destroy(AfrContext *c) {
    Range nvtx_range("afr_destroy");
    if (!c) return;
    cudaDeviceSynchronize();
    if (c->prof_ev) {
        for (int k = 0; k < 2 * AFR_PROFILE_MAX_LAUNCHES; ++k) cudaEventDestroy(c->prof_ev[k]);
        delete[] c->prof_ev;
    }
    free_all(c);
    delete c;
}

AfrStatus afr_reset(AfrContext *c, afr_stream_t stream) {
    Range nvtx_range("afr_reset");
    if (!c) return AFR_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemsetAsync(c->r_state, 0, (size_t)c->P * sizeof(uint32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->dcount, 0, afr::CNT_N * sizeof(unsigned long long), s);
    if (e == cudaSuccess && c->q_total) e = cudaMemsetAsync(c->q_total, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) return cuda_fail(c, e, "afr_reset");
    c->inserted = 0;
    c->grads_valid = c->frame_valid = c->recon_valid = false;
    c->err.clear();
    return AFR_OK;
}

static void free_batch(AfrContext *c) {
    void *ptrs[] = {c->bucket, c->fifo_flag, c->fifo_rank, c->fifo_scan};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    c->bucket = nullptr;
    c->fifo_flag = c->fifo_rank = c->fifo_scan = nullptr;
    c->batch_cap = 0;
}

AfrStatus afr_reserve(AfrContext *c, uint32_t n) {
    Range nvtx_range("afr_reserve");
    if (!c) return AFR_ERR_INVALID_ARG;
    if (n <= c->batch_cap) return AFR_OK;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(c, e, "afr_reserve");
    free_batch(c);
    e = dalloc(&c->bucket, 4 * (size_t)n);   // 64-byte records
    if (c->fifo_n) {
        if (e == cudaSuccess) e = dalloc(&c->fifo_flag, n);
        if (e == cudaSuccess) e = dalloc(&c->fifo_rank, (size_t)n + 1);   // the scan also writes the total
        if (e == cudaSuccess) e = dalloc(&c->fifo_scan, afr::scan_tmp_elems(n));
    }
    if (e != cudaSuccess) {
        free_batch(c);
        cudaGetLastError();
        return cuda_fail(c, e, "afr_reserve");
    }
    c->batch_cap = n;
    return AFR_OK;
}

static AfrStatus insert_impl(AfrContext *c, const AfrSampleBatch *batch, uint32_t n, uint32_t flags,
                             cudaEvent_t queues_free, cudaStream_t s) {
    if (!c) return AFR_ERR_INVALID_ARG;
    if (flags & ~(uint32_t)AFR_INSERT_RESET) return fail(c, AFR_ERR_INVALID_ARG, "afr_insert_samples_ex: unknown flag");
    const bool reset = (flags & AFR_INSERT_RESET) != 0;
    if (n == 0) {
        if (!reset) return AFR_OK;
        if (queues_free) {
            const cudaError_t e = cudaStreamWaitEvent(s, queues_free, 0);
            if (e != cudaSuccess) return cuda_fail(c, e, "afr_insert_samples_ex");
        }
        return afr_reset(c, reinterpret_cast<afr_stream_t>(s));
    }
    if (!batch || !batch->pos_dev || !batch->color_dev || !batch->motion_dev)
        return fail(c, AFR_ERR_INVALID_ARG, "afr_insert_samples: null batch pointer");
    if (!aligned(batch->pos_dev, 16) || !aligned(batch->color_dev, c->csize) || !aligned(batch->motion_dev, 8))
        return fail(c, AFR_ERR_INVALID_ARG, "afr_insert_samples: misaligned batch array");
    if (c->r_world && (!batch->world_dev || !aligned(batch->world_dev, 16)))
        return fail(c, AFR_ERR_INVALID_ARG, "afr_insert_samples: this context needs 16-byte aligned world points");
    const uint64_t seq0 = reset ? 0 : c->inserted;
    if (seq0 + n > 0xFFFFFFFFull)
        return fail(c, AFR_ERR_INVALID_ARG, "afr_insert_samples: sequence numbers exhausted; call afr_reset");
    AfrStatus st = afr_reserve(c, n);
    if (st != AFR_OK) return st;
    cudaError_t e = afr::launch_ingest(c, batch, n, (uint32_t)seq0, s, queues_free, reset);
    if (e == cudaSuccess && c->fifo_n) e = afr::launch_fifo_append(c, batch, n, (uint32_t)seq0, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "afr_insert_samples");
    if (reset) c->err.clear();
    c->inserted = seq0 + n;
    c->grads_valid = c->frame_valid = c->recon_valid = false;
    return AFR_OK;
}

AfrStatus afr_insert_samples(AfrContext *c, const AfrSampleBatch *batch, uint32_t n, afr_stream_t stream) {
    Range nvtx_range("afr_insert_samples");
    return insert_impl(c, batch, n, 0u, nullptr, reinterpret_cast<cudaStream_t>(stream));
}

AfrStatus afr_insert_samples_ex(AfrContext *c, const AfrSampleBatch *batch, uint32_t n, uint32_t flags,
                                afr_event_t queues_free, afr_stream_t stream) {
    Range nvtx_range("afr_insert_samples_ex");
    return insert_impl(c, batch, n, flags, reinterpret_cast<cudaEvent_t>(queues_free),
                       reinterpret_cast<cudaStream_t>(stream));
}

AfrStatus afr_estimate_gradients(AfrContext *c, float t_now, afr_stream_t stream) {
    Range nvtx_range("afr_estimate_gradients");
    if (!c) return AFR_ERR_INVALID_ARG;
    if (!std::isfinite(t_now)) return fail(c, AFR_ERR_INVALID_ARG, "afr_estimate_gradients: t_now not finite");
    cudaError_t e = afr::launch_gradients(c, t_now, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(c, e, "afr_estimate_gradients");
    c->grads_valid = true;
    c->grads_t = t_now;
    c->recon_valid = false;
    return AFR_OK;
}

AfrStatus afr_reproject_camera(AfrContext *c, float t_now, const float *view_proj, afr_stream_t stream) {
    Range nvtx_range("afr_reproject_camera");
    if (!c) return AFR_ERR_INVALID_ARG;
    if (!std::isfinite(t_now) || !view_proj)
        return fail(c, AFR_ERR_INVALID_ARG, "afr_reproject_camera: t_now not finite or null matrix");
    for (int k = 0; k < 16; ++k)
        if (!std::isfinite(view_proj[k])) return fail(c, AFR_ERR_INVALID_ARG, "afr_reproject_camera: matrix not finite");
    if (!c->r_world) return fail(c, AFR_ERR_BAD_STATE, "afr_reproject_camera: context stores no world points");
    afr::Camera cam;
    for (int k = 0; k < 4; ++k) {
        cam.m[k] = view_proj[k];           // row 0
        cam.m[4 + k] = view_proj[4 + k];   // row 1
        cam.m[8 + k] = view_proj[12 + k];  // row 3
    }
    cudaError_t e = afr::launch_reproject(c, t_now, &cam, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(c, e, "afr_reproject_camera");
    c->frame_valid = true;
    c->frame_t = t_now;
    c->recon_valid = false;
    return AFR_OK;
}

AfrStatus afr_reproject(AfrContext *c, float t_now, afr_stream_t stream) {
    Range nvtx_range("afr_reproject");
    if (!c) return AFR_ERR_INVALID_ARG;
    if (!std::isfinite(t_now)) return fail(c, AFR_ERR_INVALID_ARG, "afr_reproject: t_now not finite");
    cudaError_t e = afr::launch_reproject(c, t_now, nullptr, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(c, e, "afr_reproject");
    c->frame_valid = true;
    c->frame_t = t_now;
    c->recon_valid = false;
    return AFR_OK;
}

static bool params_ok(const AfrParams *p) {
    const float v[6] = {p->alpha_s, p->beta_s, p->clamp_s, p->alpha_t, p->beta_t, p->clamp_t};
    for (float f : v)
        if (!std::isfinite(f)) return false;
    return p->clamp_s > 0.f && p->clamp_t > 0.f;
}

AfrStatus afr_reconstruct_ex(AfrContext *c, float t_now, const AfrParams *params, uint32_t flags,
                             float *out_rgbw_dev, afr_stream_t stream) {
    Range nvtx_range("afr_reconstruct_ex");
    if (!c) return AFR_ERR_INVALID_ARG;
    if (!params || !out_rgbw_dev || !aligned(out_rgbw_dev, 16))
        return fail(c, AFR_ERR_INVALID_ARG, "afr_reconstruct: null or misaligned pointer");
    if (!params_ok(params)) return fail(c, AFR_ERR_INVALID_ARG, "afr_reconstruct: parameters not finite/positive");
    bool keep = (flags & AFR_RECON_KEEP_SIGMA) != 0;
    const bool adaptive = (flags & AFR_RECON_ADAPTIVE_SUPPORT) != 0;
    if (flags & ~(uint32_t)(AFR_RECON_KEEP_SIGMA | AFR_RECON_ADAPTIVE_SUPPORT | AFR_RECON_COVERAGE_RESET))
        return fail(c, AFR_ERR_INVALID_ARG, "afr_reconstruct_ex: unknown flag");
    if (!c->frame_valid || c->frame_t != t_now)
        return fail(c, AFR_ERR_BAD_STATE, "afr_reconstruct: call afr_reproject for this t_now first");
    if (!keep && (!c->grads_valid || c->grads_t != t_now))
        return fail(c, AFR_ERR_BAD_STATE, "afr_reconstruct: call afr_estimate_gradients for this t_now first");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (flags & AFR_RECON_COVERAGE_RESET) e = afr::launch_coverage_init(c, s);
    if (e == cudaSuccess) e = afr::launch_sigma(c, params, keep, adaptive, s);
    cudaEvent_t *pair = nullptr;
    if (e == cudaSuccess && c->prof_on && c->prof_n < AFR_PROFILE_MAX_LAUNCHES) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        e = cudaStreamIsCapturing(s, &cap);
        if (e == cudaSuccess && cap != cudaStreamCaptureStatusNone) c->prof_capture_hit = true;
        else if (e == cudaSuccess) pair = c->prof_ev + 2 * c->prof_n;
    }
    if (e == cudaSuccess && pair) e = cudaEventRecord(pair[0], s);
    if (e == cudaSuccess) e = afr::launch_filter(c, t_now, adaptive, reinterpret_cast<float4 *>(out_rgbw_dev), s);
    if (e == cudaSuccess && pair) {
        e = cudaEventRecord(pair[1], s);
        ++c->prof_n;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "afr_reconstruct");
    c->recon_valid = true;
    c->recon_t = t_now;
    c->recon_params = *params;
    c->sigma_imported = keep;
    c->adaptive_last = adaptive;
    return AFR_OK;
}

AfrStatus afr_reconstruct(AfrContext *c, float t_now, const AfrParams *params, float *out_rgbw_dev,
                          afr_stream_t stream) {
    Range nvtx_range("afr_reconstruct");
    return afr_reconstruct_ex(c, t_now, params, 0u, out_rgbw_dev, stream);
}

AfrStatus afr_tile_feedback(AfrContext *c, AfrTileStats *out_dev, afr_stream_t stream) {
    Range nvtx_range("afr_tile_feedback");
    if (!c) return AFR_ERR_INVALID_ARG;
    if (!out_dev) return fail(c, AFR_ERR_INVALID_ARG, "afr_tile_feedback: null output");
    if (!c->grads_valid) return fail(c, AFR_ERR_BAD_STATE, "afr_tile_feedback: call afr_estimate_gradients first");
    cudaError_t e = afr::launch_feedback(c, out_dev, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(c, e, "afr_tile_feedback");
    return AFR_OK;
}

AfrStatus afr_tile_error(AfrContext *c, float kappa, float lambda, float importance, const uint32_t *occluded_dev,
                         float *error_dev, AfrGain *gain_dev, afr_stream_t stream) {
    Range nvtx_range("afr_tile_error");
    if (!c) return AFR_ERR_INVALID_ARG;
    if (!error_dev) return fail(c, AFR_ERR_INVALID_ARG, "afr_tile_error: null output");
    if (!(kappa >= 0.f && lambda >= 0.f && kappa + lambda <= 1.f) || !(importance >= 0.f) || !std::isfinite(importance))
        return fail(c, AFR_ERR_INVALID_ARG, "afr_tile_error: need 0 <= kappa, lambda, kappa + lambda <= 1, importance >= 0");
    if (gain_dev && !aligned(gain_dev, 4)) return fail(c, AFR_ERR_INVALID_ARG, "afr_tile_error: misaligned gain");
    if (!c->grads_valid) return fail(c, AFR_ERR_BAD_STATE, "afr_tile_error: call afr_estimate_gradients first");
    cudaError_t e = afr::launch_tile_error(c, kappa, lambda, importance, occluded_dev, error_dev, gain_dev,
                                           reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(c, e, "afr_tile_error");
    return AFR_OK;
}

AfrStatus afr_reconstruct_backward(AfrContext *c, const float *grad_rgb_dev, float *grad_colors_dev,
                                   float *grad_params_dev, afr_stream_t stream) {
    Range nvtx_range("afr_reconstruct_backward");
    if (!c) return AFR_ERR_INVALID_ARG;
    if (!grad_rgb_dev || !aligned(grad_rgb_dev, 16))
        return fail(c, AFR_ERR_INVALID_ARG, "afr_reconstruct_backward: null or misaligned grad_rgb");
    if (!c->recon_valid || !c->frame_valid)
        return fail(c, AFR_ERR_BAD_STATE, "afr_reconstruct_backward: call afr_reconstruct first");
    if (c->adaptive_last)
        return fail(c, AFR_ERR_BAD_STATE, "afr_reconstruct_backward: not available after an adaptive reconstruction");
    if (grad_params_dev && (c->sigma_imported || !c->grads_valid))
        return fail(c, AFR_ERR_BAD_STATE,
                    "afr_reconstruct_backward: parameter gradients need widths computed from gradients");
    cudaError_t e = afr::launch_backward(c, reinterpret_cast<const float4 *>(grad_rgb_dev), grad_colors_dev,
                                         grad_params_dev, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(c, e, "afr_reconstruct_backward");
    return AFR_OK;
}

AfrStatus afr_get_status(AfrContext *c, afr_stream_t stream) {
    if (!c) return AFR_ERR_INVALID_ARG;
    Range r("afr_get_status");
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    uint32_t w = 0;
    cudaError_t e = cudaMemcpyAsync(&w, c->derr, sizeof(w), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "afr_get_status");
    if (w) {
        e = cudaMemsetAsync(c->derr, 0, sizeof(uint32_t), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(c, e, "afr_get_status");
        if (w & afr::ERR_TIMEOUT) return fail(c, AFR_ERR_TIMEOUT, "a bounded device-side wait ran out");
        return fail(c, AFR_ERR_DEVICE_CHECK, "a device-side check failed");
    }
    return AFR_OK;
}

const char *afr_last_error(const AfrContext *c) { return c ? c->err.c_str() : "null context"; }

AfrStatus afr_query(AfrContext *c, AfrInfo *info, afr_stream_t stream) {
    Range nvtx_range("afr_query");
    if (!c || !info) return AFR_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = afr::launch_resident_count(c, s);
    unsigned long long cnt[afr::CNT_N] = {0};
    uint32_t frame = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, c->dcount, sizeof(cnt), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&frame, c->foff + c->P, sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "afr_query");
    info->inserted = c->inserted;
    info->rejected = cnt[afr::CNT_REJECTED];
    info->resident = cnt[afr::CNT_RESIDENT];
    info->frame = c->frame_valid ? frame : 0;
    info->dropped = cnt[afr::CNT_DROPPED];
    info->unsorted_bins = cnt[afr::CNT_UNSORTED];
    return AFR_OK;
}

AfrStatus afr_num_tiles(const AfrContext *c, uint32_t *n) {
    Range nvtx_range("afr_num_tiles");
    if (!c || !n) return AFR_ERR_INVALID_ARG;
    *n = (uint32_t)c->ntiles;
    return AFR_OK;
}

AfrStatus afr_export_ring(AfrContext *c, int32_t *count_host, float *slot_host, uint32_t *seq_host) {
    Range nvtx_range("afr_export_ring");
    if (!c || !count_host || !slot_host || !seq_host) return AFR_ERR_INVALID_ARG;
    size_t P = c->P, N = c->nslots;
    std::vector<uint32_t> state(P), seq(N);
    std::vector<float2> xy(N), mo(N);
    std::vector<float> t(N), depth(N);
    std::vector<unsigned char> col(N * c->csize);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(state.data(), c->r_state, P * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(seq.data(), c->r_seq, N * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(xy.data(), c->r_xy, N * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(mo.data(), c->r_mo, N * 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(t.data(), c->r_t, N * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(depth.data(), c->r_depth, N * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(col.data(), c->r_col, N * c->csize, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "afr_export_ring");
    std::memset(slot_host, 0, N * 9 * sizeof(float));
    std::memset(seq_host, 0, N * sizeof(uint32_t));
    for (size_t p = 0; p < P; ++p) {
        int n = (int)(state[p] & 0xFFFFu), h = (int)(state[p] >> 16);
        count_host[p] = n;
        for (int k = 0; k < n; ++k) {
            int s = h - 1 - k;
            if (s < 0) s += c->b;
            size_t i = p * c->b + s;
            float *o = slot_host + (p * c->b + k) * 9;
            o[0] = xy[i].x;
            o[1] = xy[i].y;
            o[2] = t[i];
            o[3] = depth[i];
            widen_colors(c->ct, col.data(), i, o + 4);
            o[7] = mo[i].x;
            o[8] = mo[i].y;
            seq_host[p * c->b + k] = seq[i];
        }
    }
    return AFR_OK;
}

AfrStatus afr_export_frame(AfrContext *c, uint32_t *off_host, float *rec_host, uint32_t *seq_host, uint64_t cap) {
    Range nvtx_range("afr_export_frame");
    if (!c || !off_host || !rec_host || !seq_host) return AFR_ERR_INVALID_ARG;
    if (!c->frame_valid) return fail(c, AFR_ERR_BAD_STATE, "afr_export_frame: no frame view");
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(off_host, c->foff, (size_t)(c->P + 1) * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "afr_export_frame");
    size_t n = off_host[c->P];
    if (n > cap) return fail(c, AFR_ERR_INVALID_ARG, "afr_export_frame: capacity too small");
    std::vector<float4> pos(n ? n : 1);
    std::vector<unsigned char> col((n ? n : 1) * c->csize);
    if (n) {
        e = cudaMemcpy(pos.data(), c->fpos, n * 16, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(col.data(), c->fcol, n * c->csize, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(seq_host, c->fseq, n * 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, "afr_export_frame");
    }
    for (size_t i = 0; i < n; ++i) {
        float *o = rec_host + i * 6;
        o[0] = pos[i].x;
        o[1] = pos[i].y;
        o[2] = pos[i].z;
        widen_colors(c->ct, col.data(), i, o + 3);
    }
    return AFR_OK;
}

AfrStatus afr_export_map(AfrContext *c, AfrMap which, float *map_host) {
    Range nvtx_range("afr_export_map");
    if (!c || !map_host) return AFR_ERR_INVALID_ARG;
    size_t P = c->P;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(c, e, "afr_export_map");
    if (which == AFR_MAP_LBAR) {   // the high part of the double-float mean
        e = cudaMemcpy2D(map_host, 4, c->lbar, 8, 4, P, cudaMemcpyDeviceToHost);
    } else if (which >= AFR_MAP_GX && which <= AFR_MAP_GT) {
        e = cudaMemcpy2D(map_host, 4, reinterpret_cast<float *>(c->grad) + (which - AFR_MAP_GX), 16, 4, P,
                         cudaMemcpyDeviceToHost);
    } else if (which == AFR_MAP_SIGMA_S || which == AFR_MAP_SIGMA_T) {
        e = cudaMemcpy2D(map_host, 4, reinterpret_cast<float *>(c->sigma) + (which - AFR_MAP_SIGMA_S), 8, 4, P,
                         cudaMemcpyDeviceToHost);
    } else if (which == AFR_MAP_FOOTPRINT) {
        e = cudaMemcpy(map_host, c->cov_r[c->cov_cur], P * 4, cudaMemcpyDeviceToHost);
    } else if (which == AFR_MAP_COVERAGE) {
        std::vector<int32_t> n(P);
        e = cudaMemcpy(n.data(), c->cov_n, P * 4, cudaMemcpyDeviceToHost);
        for (size_t p = 0; p < P && e == cudaSuccess; ++p) map_host[p] = (float)n[p];
    } else {
        return fail(c, AFR_ERR_INVALID_ARG, "afr_export_map: unknown map");
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "afr_export_map");
    return AFR_OK;
}

AfrStatus afr_import_map(AfrContext *c, AfrMap which, const float *map_host) {
    Range nvtx_range("afr_import_map");
    if (!c || !map_host) return AFR_ERR_INVALID_ARG;
    size_t P = c->P;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(c, e, "afr_import_map");
    if (which == AFR_MAP_LBAR) {   // imported means have no low part
        e = cudaMemset(c->lbar, 0, P * sizeof(float2));
        if (e == cudaSuccess) e = cudaMemcpy2D(c->lbar, 8, map_host, 4, 4, P, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy2D(reinterpret_cast<float *>(c->grad) + 3, 16, map_host, 4, 4, P, cudaMemcpyHostToDevice);
    } else if (which >= AFR_MAP_GX && which <= AFR_MAP_GT) {
        e = cudaMemcpy2D(reinterpret_cast<float *>(c->grad) + (which - AFR_MAP_GX), 16, map_host, 4, 4, P,
                         cudaMemcpyHostToDevice);
    } else if (which == AFR_MAP_SIGMA_S || which == AFR_MAP_SIGMA_T) {
        e = cudaMemcpy2D(reinterpret_cast<float *>(c->sigma) + (which - AFR_MAP_SIGMA_S), 8, map_host, 4, 4, P,
                         cudaMemcpyHostToDevice);
    } else {
        return fail(c, AFR_ERR_INVALID_ARG, "afr_import_map: unknown map");
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "afr_import_map");
    c->recon_valid = false;
    return AFR_OK;
}

AfrStatus afr_set_frame_colors(AfrContext *c, const float *rgb_dev, afr_stream_t stream) {
    Range nvtx_range("afr_set_frame_colors");
    if (!c || !rgb_dev) return AFR_ERR_INVALID_ARG;
    if (!c->frame_valid) return fail(c, AFR_ERR_BAD_STATE, "afr_set_frame_colors: no frame view");
    cudaError_t e = afr::launch_set_frame_colors(c, rgb_dev, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(c, e, "afr_set_frame_colors");
    c->recon_valid = false;
    return AFR_OK;
}

}  // extern "C"

extern "C" {

AfrStatus afr_profile_filter(AfrContext *c, int32_t enable) {
    Range nvtx_range("afr_profile_filter");
    if (!c) return AFR_ERR_INVALID_ARG;
    if (enable && !c->prof_ev) {
        c->prof_ev = new cudaEvent_t[2 * AFR_PROFILE_MAX_LAUNCHES]();
        for (int k = 0; k < 2 * AFR_PROFILE_MAX_LAUNCHES; ++k) {
            cudaError_t e = cudaEventCreate(&c->prof_ev[k]);
            if (e != cudaSuccess) {
                for (int j = 0; j < k; ++j) cudaEventDestroy(c->prof_ev[j]);
                delete[] c->prof_ev;
                c->prof_ev = nullptr;
                return cuda_fail(c, e, "afr_profile_filter");
            }
        }
    }
    if (enable) {
        c->prof_n = 0;
        c->prof_capture_hit = false;
    }
    c->prof_on = enable != 0;
    return AFR_OK;
}

AfrStatus afr_profile_read(AfrContext *c, float *ms, int32_t cap, int32_t *count) {
    Range nvtx_range("afr_profile_read");
    if (!c || !count || (cap > 0 && !ms) || cap < 0) return AFR_ERR_INVALID_ARG;
    *count = 0;
    const int n = c->prof_n;
    for (int k = 0; k < n; ++k) {
        cudaError_t e = cudaEventSynchronize(c->prof_ev[2 * k + 1]);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, c->prof_ev[2 * k], c->prof_ev[2 * k + 1]);
        if (e != cudaSuccess) return cuda_fail(c, e, "afr_profile_read");
        if (k < cap) ms[k] = t;
    }
    *count = n;
    c->prof_n = 0;
    const bool hit = c->prof_capture_hit;
    c->prof_capture_hit = false;
    if (hit) return fail(c, AFR_ERR_BAD_STATE, "afr_profile_read: launches under stream capture were not timed");
    return AFR_OK;
}

AfrStatus afr_set_tuning(AfrContext *c, int32_t radius, int32_t tile_bx) {
    Range nvtx_range("afr_set_tuning");
    if (!c) return AFR_ERR_INVALID_ARG;
    if (radius < 0 || radius > 8 || !(tile_bx == 2 || tile_bx == 4 || tile_bx == 8 || tile_bx == 16))
        return fail(c, AFR_ERR_INVALID_ARG, "afr_set_tuning: radius 0..8, tile_bx 2, 4, 8 or 16");
    c->R = radius;
    c->cfg.radius = radius;
    c->tile_bx = tile_bx;
    c->recon_valid = false;
    return AFR_OK;
}

void afr_batch_destroy(AfrBatch *b) {
    Range nvtx_range("afr_batch_destroy");
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->h_ctx) cudaFreeHost(b->h_ctx);
    if (b->d_ctx) cudaFree(b->d_ctx);
    if (b->d_queue) cudaFree(b->d_queue);
    for (cudaStream_t w : b->workers) cudaStreamDestroy(w);
    for (cudaEvent_t e : b->joined) cudaEventDestroy(e);
    if (b->forked) cudaEventDestroy(b->forked);
    delete b;
}

AfrStatus afr_batch_create(AfrContext *const *ctxs, int32_t n, AfrBatch **out) {
    Range nvtx_range("afr_batch_create");
    if (!ctxs || !out || n < 1 || n > 64) return AFR_ERR_INVALID_ARG;
    *out = nullptr;
    for (int i = 0; i < n; ++i)
        if (!ctxs[i] || ctxs[i]->ct != ctxs[0]->ct) return AFR_ERR_INVALID_ARG;
    AfrBatch *b = new (std::nothrow) AfrBatch();
    if (!b) return AFR_ERR_OOM;
    b->ct = ctxs[0]->ct;
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return ctxs[a]->P > ctxs[c]->P; });
    for (int i : order) {
        b->ctxs.push_back(ctxs[i]);
        b->user_index.push_back(i);
        b->tile_bx.push_back(ctxs[i]->tile_bx);
    }
    cudaError_t e = cudaMallocHost(&b->h_ctx, sizeof(afr::BatchCtx) * n);
    if (e == cudaSuccess) e = dmalloc(reinterpret_cast<void **>(&b->d_ctx), sizeof(afr::BatchCtx) * n);
    if (e == cudaSuccess) e = dmalloc(reinterpret_cast<void **>(&b->d_queue), sizeof(uint32_t));
    // Contexts larger than afr::kBatchDirectPixels are reconstructed with their
    // own launches inside the batched call: measured on GB300, the persistent
    // kernel is about 30% faster than separate launches for 256x256 streams
    // and 5-12% slower from 640x480 up, where each launch fills the GPU.
    while (b->n_direct < n && b->ctxs[b->n_direct]->P > afr::kBatchDirectPixels) ++b->n_direct;
    uint32_t f = 0, chunks = 0;
    for (int q = b->n_direct; q < n && e == cudaSuccess; ++q) {
        AfrContext *c = b->ctxs[q];
        const int tw = 2 * b->tile_bx[q], th = 2 * (32 / b->tile_bx[q]);
        const uint32_t bands = (uint32_t)((c->H + th - 1) / th), tx = (uint32_t)((c->W + tw - 1) / tw);
        b->h_ctx[q].a0 = f;
        b->h_ctx[q].s0 = chunks;
        f += bands * tx;
        chunks += (uint32_t)((c->P + afr::kBatchSigmaChunk - 1) / afr::kBatchSigmaChunk);
    }
    b->total = f;
    b->nchunks = chunks;
    int dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        afr_batch_destroy(b);
        return e == cudaErrorMemoryAllocation ? AFR_ERR_OOM : AFR_ERR_CUDA;
    }
    b->grid = 3 * sms;
    // afr_batch_refresh: kBatchWorkers streams, each context on the one with
    // the least work so far (work ~ its buffered slots), largest first
    const int nw = std::min(n, afr::kBatchWorkers);
    std::vector<double> load(nw, 0.0);
    for (int q = 0; q < n; ++q) {
        const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        b->worker_of.push_back(w);
        load[w] += (double)b->ctxs[q]->P * (b->ctxs[q]->b + 8);
    }
    for (int w = 0; w < nw && e == cudaSuccess; ++w) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) b->workers.push_back(st);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e == cudaSuccess) b->joined.push_back(ev);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->forked, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        afr_batch_destroy(b);
        return AFR_ERR_CUDA;
    }
    *out = b;
    return AFR_OK;
}


AfrStatus afr_batch_refresh(AfrBatch *b, float t_now, const AfrParams *params, float *const *outs_dev,
                            afr_stream_t stream) {
    Range nvtx_range("afr_batch_refresh");
    if (!b || !params || !outs_dev || !std::isfinite(t_now)) return AFR_ERR_INVALID_ARG;
    if (!params_ok(params)) return AFR_ERR_INVALID_ARG;
    const int n = (int)b->ctxs.size();
    for (int q = 0; q < n; ++q) {
        float *o = outs_dev[b->user_index[q]];
        if (!o || !aligned(o, 16))
            return fail(b->ctxs[q], AFR_ERR_INVALID_ARG, "afr_batch_refresh: bad output pointer");
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaEventRecord(b->forked, s);
    for (size_t w = 0; w < b->workers.size() && e == cudaSuccess; ++w) e = cudaStreamWaitEvent(b->workers[w], b->forked, 0);
    for (int q = 0; q < n && e == cudaSuccess; ++q) {
        AfrContext *c = b->ctxs[q];
        cudaStream_t ws = b->workers[b->worker_of[q]];
        e = afr::launch_gradients(c, t_now, ws);
        if (e == cudaSuccess) e = afr::launch_reproject(c, t_now, nullptr, ws);
        if (e == cudaSuccess) e = afr::launch_sigma(c, params, false, false, ws);
        if (e == cudaSuccess)
            e = afr::launch_filter(c, t_now, false, reinterpret_cast<float4 *>(outs_dev[b->user_index[q]]), ws);
    }
    for (size_t w = 0; w < b->workers.size() && e == cudaSuccess; ++w) {
        e = cudaEventRecord(b->joined[w], b->workers[w]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->joined[w], 0);
    }
    if (e != cudaSuccess) return cuda_fail(b->ctxs[0], e, "afr_batch_refresh");
    for (AfrContext *c : b->ctxs) {
        c->grads_valid = c->frame_valid = c->recon_valid = true;
        c->grads_t = c->frame_t = c->recon_t = t_now;
        c->recon_params = *params;
        c->sigma_imported = false;
        c->adaptive_last = false;
    }
    return AFR_OK;
}

AfrStatus afr_batch_reconstruct(AfrBatch *b, float t_now, const AfrParams *params, float *const *outs_dev,
                                afr_stream_t stream) {
    Range nvtx_range("afr_batch_reconstruct");
    if (!b || !params || !outs_dev) return AFR_ERR_INVALID_ARG;
    if (!params_ok(params)) return AFR_ERR_INVALID_ARG;
    const int n = (int)b->ctxs.size();
    std::vector<afr::BatchCtx> rec(b->h_ctx, b->h_ctx + n);
    for (int q = 0; q < n; ++q) {
        AfrContext *c = b->ctxs[q];
        float *o = outs_dev[b->user_index[q]];
        if (!o || !aligned(o, 16)) return fail(c, AFR_ERR_INVALID_ARG, "afr_batch_reconstruct: bad output pointer");
        if (!c->frame_valid || c->frame_t != t_now || !c->grads_valid || c->grads_t != t_now)
            return fail(c, AFR_ERR_BAD_STATE, "afr_batch_reconstruct: estimate gradients and reproject first");
        if (c->tile_bx != b->tile_bx[q])
            return fail(c, AFR_ERR_BAD_STATE, "afr_batch_reconstruct: tile shape changed since afr_batch_create");
        afr::BatchCtx &x = rec[q];
        x.W = c->W;
        x.H = c->H;
        x.R = c->R;
        x.S = c->S;
        x.ntx = c->ntx;
        x.tbx = c->tile_bx;
        x.th = 2 * (32 / c->tile_bx);
        x.ntiles_x = (c->W + 2 * c->tile_bx - 1) / (2 * c->tile_bx);
        x.window = c->cfg.window;
        x.eps = c->cfg.eps_grad;
        x.prm = *params;
        x.grad = c->grad;
        x.tiles = c->tiles;
        x.sigma = c->sigma;
        x.fconst = c->fconst;
        x.amin2 = c->amin2;
        x.foff = c->foff;
        x.fpos = c->fpos;
        x.fcol = c->fcol;
        x.out = reinterpret_cast<float4 *>(o);
        x.derr = c->derr;
        x.fcap = (uint32_t)c->frame_cap;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // the pinned staging buffer may still feed an earlier copy on the stream:
    // rewrite it only when the records change, after the stream drains (a
    // stream being captured has nothing in flight)
    if (std::memcmp(rec.data(), b->h_ctx, sizeof(afr::BatchCtx) * n) != 0) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        cudaError_t ce = cudaStreamIsCapturing(s, &cap);
        if (ce == cudaSuccess && cap == cudaStreamCaptureStatusNone) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) return cuda_fail(b->ctxs[0], ce, "afr_batch_reconstruct");
        std::memcpy(b->h_ctx, rec.data(), sizeof(afr::BatchCtx) * n);
    }
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < b->n_direct && e == cudaSuccess; ++q) {
        AfrContext *c = b->ctxs[q];
        e = afr::launch_sigma(c, params, false, false, s);
        if (e == cudaSuccess)
            e = afr::launch_filter(c, t_now, false, reinterpret_cast<float4 *>(outs_dev[b->user_index[q]]), s);
    }
    const int m = n - b->n_direct;
    if (m > 0) {
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_ctx + b->n_direct, b->h_ctx + b->n_direct, sizeof(afr::BatchCtx) * m,
                                cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(b->d_queue, 0, sizeof(uint32_t), s);
        if (e == cudaSuccess)
            e = afr::launch_batch(b->ct, b->d_ctx + b->n_direct, m, b->nchunks, b->total, b->d_queue, b->grid, s);
    }
    if (e != cudaSuccess) return cuda_fail(b->ctxs[0], e, "afr_batch_reconstruct");
    for (AfrContext *c : b->ctxs) {
        c->recon_valid = true;
        c->recon_t = t_now;
        c->recon_params = *params;
        c->sigma_imported = false;
        c->adaptive_last = false;
    }
    return AFR_OK;
}

}  // extern "C"

#ifdef AFR_DEBUG
extern "C" {

void afr_debug_fail_alloc(int32_t after) {
    g_fail_after = after;
    g_allocs = 0;
}

AfrStatus afr_debug_set_frame_offsets(AfrContext *c, const uint32_t *off_host) {
    if (!c || !off_host) return AFR_ERR_INVALID_ARG;
    for (int p = 0; p < c->P; ++p)
        if (off_host[p + 1] < off_host[p]) return fail(c, AFR_ERR_INVALID_ARG, "offsets must not decrease");
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(c->foff, off_host, sizeof(uint32_t) * ((size_t)c->P + 1), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(c, e, "afr_debug_set_frame_offsets");
    return AFR_OK;
}

}  // extern "C"
#endif

/*
 * afr.h -- C ABI of the GB300 reconstruction path of adaptive frameless
 * rendering (Dayal, Woolley, Watson and Luebke, "Adaptive Frameless
 * Rendering").
 *
 * The library keeps, per context, the reconstructor's temporally deep buffer
 * (section 4: a per-pixel queue of depth b), estimates space-time colour
 * gradients from it (section 4.1), reprojects the buffered samples to the
 * display time (section 6.2), filters every pixel with a space-time Gaussian
 * whose widths follow local sample density and gradients (sections 5.1 and
 * 5.2), returns per-tile statistics for the sampler (sections 4, 4.2, 6.1)
 * and runs the adjoint of the filter for fitting its width mapping.
 *
 * Conventions shared by every entry point:
 *  - Pointers named *_dev are device memory owned by the caller; pointers
 *    named *_host are host memory owned by the caller. The context owns its
 *    internal buffers and frees them in afr_destroy.
 *  - Compute calls are asynchronous on the given stream and return argument
 *    or call-order errors synchronously. Failures detected on the device
 *    (a failed internal check of a debug build, see afr_debug.h) are recorded
 *    in a device status word that afr_get_status reads (it synchronises the
 *    stream it is given).
 *  - Nothing throws across the ABI and there is no CPU fallback: when no
 *    CUDA device is usable, afr_create returns AFR_ERR_CUDA.
 *  - Calls on one context are not thread-safe; distinct contexts are
 *    independent.
 *  - After afr_insert_samples, afr_estimate_gradients (with the
 *    afr_tile_feedback and afr_tile_error that read its tile statistics) and
 *    afr_reproject or afr_reproject_camera read the sample buffers and write
 *    disjoint state, so the two branches may be issued on two streams and run
 *    concurrently; afr_reconstruct reads both branches' results and must be
 *    ordered after both (for instance with an event recorded on the other
 *    stream). afr_reconstruct reads neither the sample buffers nor the ingest
 *    scratch, so the next afr_reset and afr_insert_samples may run on another
 *    stream concurrently with it, once both branches have finished; the next
 *    afr_estimate_gradients and afr_reproject must again follow it. (The call
 *    order checks are made when a call is issued: issue afr_reconstruct before
 *    the next afr_insert_samples.)
 */
#ifndef AFR_H
#define AFR_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define AFR_API __attribute__((visibility("default")))
#else
#define AFR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as the CUDA runtime's cudaStream_t; 0 is the legacy stream. */
typedef struct CUstream_st *afr_stream_t;
/* Same type as the CUDA runtime's cudaEvent_t. */
typedef struct CUevent_st *afr_event_t;

typedef enum {
    AFR_OK = 0,
    AFR_ERR_INVALID_ARG = 1,   /* a pointer, size or parameter out of range */
    AFR_ERR_BAD_STATE = 2,     /* calls out of order (see each call) */
    AFR_ERR_OOM = 3,           /* a device allocation failed */
    AFR_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    AFR_ERR_TIMEOUT = 5,       /* reserved: a bounded device-side wait ran out (no call waits) */
    AFR_ERR_DEVICE_CHECK = 6   /* a device-side consistency check failed */
} AfrStatus;

/* Storage type of buffered sample colours. Accumulation is always FP32. */
typedef enum { AFR_F32 = 0, AFR_F16 = 1, AFR_BF16 = 2 } AfrColorType;

typedef struct {
    int32_t width, height;   /* image size in pixels, 1..16384 each */
    int32_t depth;           /* b, queue depth per pixel, 1..32 (section 4 uses 4);
                                width*height*depth must not exceed 2^28 */
    int32_t tile;            /* S, side of the density/statistics tiles, 1..256 (default 32) */
    int32_t radius;          /* R, filter footprint radius in bins, 0..8 (default 4) */
    int32_t color_type;      /* AfrColorType */
    float window;            /* length of the time window in its own units (default 1) */
    float eps_grad;          /* floor of the gradients in the extent rule (default 1e-4) */
    float undersample_m;     /* m of the undersampling measure (default 2) */
    uint32_t fifo_capacity;  /* section 5.2: 0 (default) reprojects the per-pixel queues; N > 0
                                also keeps the N most recent accepted samples of the whole
                                image in one queue, and afr_reproject builds the frame view
                                from that queue instead (N <= 2^28) */
    uint32_t world_points;   /* section 6.2: nonzero if every sample carries the 3D hit point of its
                                primary ray (AfrSampleBatch.world_dev), which the context stores
                                for afr_reproject_camera */
} AfrConfig;

/* Mapping from filter extents to Gaussian widths (theta). Section 5.1 sizes
 * the extents; the widths are sigma_s = min(max(alpha_s e_s + beta_s, 0.5),
 * clamp_s) in pixels and sigma_t = min(max(alpha_t e_t + beta_t, 0.05),
 * clamp_t) in window units. Defaults 1, 0, 3, 1, 0, 1. */
typedef struct {
    float alpha_s, beta_s, clamp_s, alpha_t, beta_t, clamp_t;
} AfrParams;

/* One batch of samples in device memory, sample i in insertion order:
 *   pos_dev[i]    float4 (x, y, t, depth): pixel units, t in window units
 *   color_dev[i]  4 x float32 (r, g, b, unused) for AFR_F32 contexts, or
 *                 4 x 16-bit (r, g, b, unused) in the context's colour type
 *   motion_dev[i] float2 screen velocity in pixels per window
 * Each array must be 16-byte aligned (8-byte for motion and 16-bit colours). */
typedef struct {
    const void *pos_dev;
    const void *color_dev;
    const void *motion_dev;
    const void *world_dev;   /* float4 (X, Y, Z, unused) hit point per sample, 16-byte aligned;
                                required by contexts created with world_points, else ignored */
} AfrSampleBatch;

/* Per-tile statistics (sections 4, 4.2 and 6.1), tiles row-major over a
 * ceil(height/S) x ceil(width/S) grid. */
typedef struct {
    uint32_t n;            /* buffered samples whose pixel lies in the tile */
    uint32_t empty_slots;  /* tile pixels * b - n */
    float mean_L;          /* age-weighted mean luminance (0 if n == 0) */
    float var_L;           /* age-weighted luminance variance */
    float mean_Gx, mean_Gy, mean_Gt;  /* mean gradients over non-empty pixels */
    float u;               /* undersampling measure */
} AfrTileStats;

/* Counters read back by afr_query (synchronises the stream). */
typedef struct {
    uint64_t inserted;     /* samples offered to afr_insert_samples so far */
    uint64_t rejected;     /* of those, rejected (non-finite or off-image) */
    uint64_t resident;     /* samples in the deep buffer now */
    uint64_t frame;        /* samples in the frame view of the last afr_reproject */
    uint64_t dropped;      /* samples the last afr_reproject moved off-image */
    uint64_t unsorted_bins;/* frame bins too full to order by sequence (see afr_reproject) */
} AfrInfo;

typedef struct AfrContext AfrContext;

/* Creates a context on the current CUDA device and allocates its buffers
 * (deep buffer, gradient and width maps, frame view sized for width*height*
 * depth samples, tile records). Returns AFR_ERR_INVALID_ARG for a config out
 * of range, AFR_ERR_OOM / AFR_ERR_CUDA on failure (nothing is leaked). */
AFR_API AfrStatus afr_create(const AfrConfig *cfg, AfrContext **out);

/* Frees everything the context owns. Safe on NULL. Synchronises the device. */
AFR_API void afr_destroy(AfrContext *ctx);

/* Empties the deep buffer (and the reconstructor's queue of a context with
 * fifo_capacity > 0) and restarts sequence numbering. */
AFR_API AfrStatus afr_reset(AfrContext *ctx, afr_stream_t stream);

/* Grows the context's ingest scratch to hold batches of up to n samples so
 * that later afr_insert_samples calls do not allocate. */
AFR_API AfrStatus afr_reserve(AfrContext *ctx, uint32_t n);

/* Section 4 (deep buffer): pushes n samples, in index order, into the
 * queues of the pixels that contain them. A sample whose x, y, t, colour or
 * motion is not finite, or whose position lies outside [0,width) x
 * [0,height), is rejected and counted. A queue keeps its b newest samples by
 * insertion order; sample i of the batch gets sequence number
 * inserted_so_far + i. Grows the ingest scratch if n exceeds what
 * afr_reserve set aside (that growth allocates and synchronises).
 * Invalidates gradients and the frame view. n = 0 is a no-op. */
AFR_API AfrStatus afr_insert_samples(AfrContext *ctx, const AfrSampleBatch *batch, uint32_t n,
                             afr_stream_t stream);

/* afr_insert_samples (section 4) with two options for pipelined image loops.
 *   flags        AFR_INSERT_RESET: the queues, the reconstructor queue and the
 *                counters are cleared before the batch enters them, as
 *                afr_reset followed by afr_insert_samples would do (the
 *                batch's sequence numbers start at 0).
 *   queues_free  a CUDA event (cudaEvent_t) or NULL. The steps that read or
 *                write the queues (the reset, the copy of the queue states,
 *                the commit, the reconstructor-queue append) first wait for
 *                it on the stream; the binning before them (counting, bucket
 *                offsets, the 64-byte bucket records: scratch of this
 *                context) does not. Recorded when the previous image's
 *                afr_estimate_gradients and afr_reproject are done with the
 *                queues, it lets the next batch's binning run beside them.
 *                The event must have been recorded when the call is made.
 * The result equals afr_insert_samples (after afr_reset with the flag) bit
 * for bit. Errors as afr_insert_samples; unknown flags: AFR_ERR_INVALID_ARG. */
#define AFR_INSERT_RESET 1u
AFR_API AfrStatus afr_insert_samples_ex(AfrContext *ctx, const AfrSampleBatch *batch, uint32_t n, uint32_t flags,
                                        afr_event_t queues_free, afr_stream_t stream);

/* Sections 4 and 4.1: per-pixel age-weighted mean luminance (weights
 * exp(-3.47 a), a = max(0, t_now - t)), spatial gradients G_x, G_y (mean of
 * the one-sided absolute luminance differences to the existing non-empty
 * neighbours) and temporal gradient G_t (over the pixel's queue ordered by
 * time, newest first: age-weighted sum of |dL| over consecutive samples
 * divided by the age-weighted sum of their time steps), plus the per-tile
 * partial statistics that afr_tile_feedback and afr_reconstruct read. */
AFR_API AfrStatus afr_estimate_gradients(AfrContext *ctx, float t_now, afr_stream_t stream);

/* Section 6.2: moves every buffered sample (with fifo_capacity N > 0: every
 * sample of the reconstructor's queue of the N most recent accepted samples,
 * section 5.2) to t_now along its motion,
 * x' = x + m_x (t_now - t) in single precision with one rounding per
 * operation, and bins it at the pixel holding x' into the frame view.
 * Samples leaving the image are dropped and counted. Within a bin, records
 * are ordered by sequence number; a bin holding more than 4096 records keeps
 * arrival order instead (counted in AfrInfo.unsorted_bins). */
AFR_API AfrStatus afr_reproject(AfrContext *ctx, float t_now, afr_stream_t stream);

/* Section 6.2 with camera matrices: the frame view for t_now built by
 * rendering every buffered sample's stored 3D hit point (X, Y, Z) with the
 * current camera, view_proj_host (16 floats, row-major, host memory): with
 * c = view_proj (X, Y, Z, 1) (each row summed left to right),
 * x' = (c_x / c_w * 1/2 + 1/2) width + m_x (t_now - t) and
 * y' = (c_y / c_w * 1/2 + 1/2) height + m_y (t_now - t), where m is the
 * sample's own screen motion (zero for static geometry), in single precision
 * with one rounding per operation. Samples with c_w <= 0 or leaving the image
 * are dropped and counted; the rest are binned as afr_reproject bins them
 * (from the reconstructor queue when fifo_capacity > 0). Requires a context
 * created with world_points (else AFR_ERR_BAD_STATE). */
AFR_API AfrStatus afr_reproject_camera(AfrContext *ctx, float t_now, const float *view_proj_host,
                                       afr_stream_t stream);

/* Sections 5.1 and 5.2: for every pixel, the extents e_s = cbrt(V_S G_t/G_s),
 * e_t = cbrt(V_S G_s^2/G_t^2) (V_S = tile pixels * window / tile samples,
 * G_s = max((G_x+G_y)/2, eps), G_t floored at eps), the widths of AfrParams,
 * and the normalised Gaussian-weighted mean of the frame-view samples whose
 * bins lie within the integer disc of radius R around the pixel's bin:
 * w = exp(-|x' - c|^2 / (2 sigma_s^2) - (t_now - t)^2 / (2 sigma_t^2)).
 * out_rgbw_dev receives width*height float4 (r, g, b, W) row-major, W the
 * weight sum; a pixel with no sample in its footprint gets (0, 0, 0, 0).
 * Requires afr_estimate_gradients and afr_reproject for this t_now since the
 * last insertion (else AFR_ERR_BAD_STATE). */
AFR_API AfrStatus afr_reconstruct(AfrContext *ctx, float t_now, const AfrParams *params,
                          float *out_rgbw_dev, afr_stream_t stream);

/* Sections 4, 4.2, 6.1: writes one AfrTileStats per tile to out_dev, with
 * u = 1 - min(1, m * mean_empty / empty) (0 for a tile with no empty slot).
 * Requires afr_estimate_gradients since the last insertion. */
AFR_API AfrStatus afr_tile_feedback(AfrContext *ctx, AfrTileStats *out_dev, afr_stream_t stream);

/* Sections 6.1 and 4.1: the sampler's tile error and gain control, from the
 * tile statistics of the last afr_estimate_gradients (afr_tile_feedback need
 * not be called first). error_dev (device, n_tiles floats, required) gets
 * E_t = s_t (kappa v_t / sum v + lambda u_t / sum u
 *            + (1 - kappa - lambda) o_t / sum o),
 * s_t the tile's pixel count, v_t the age-weighted luminance variance, u_t
 * the undersampling measure, o_t = occluded_t / (s_t b) from occluded_dev
 * (device, n_tiles counts of occluded samples found by the caller's own
 * occlusion test; NULL: no occlusion data); a term whose sum over tiles is 0
 * adds 0. gain_dev (device, may be NULL) gets the gain control: the image
 * means over non-empty pixels of (G_x + G_y) / 2 and of G_t, the mean over
 * tiles holding samples of their mean sample age, the tile width S* =
 * importance dC/dt T / max(dC/ds, eps_grad) that balances spatial and
 * temporal change (dC/ds S = i dC/dt T), and the tile count W H / S*^2
 * clamped to [1, W H]. Requires 0 <= kappa, lambda and kappa + lambda <= 1,
 * importance >= 0 (else AFR_ERR_INVALID_ARG). */
typedef struct {
    float dC_ds, dC_dt, mean_age, tile_width, tile_count;
} AfrGain;
AFR_API AfrStatus afr_tile_error(AfrContext *ctx, float kappa, float lambda, float importance,
                                 const uint32_t *occluded_dev, float *error_dev, AfrGain *gain_dev,
                                 afr_stream_t stream);

/* Adjoint of afr_reconstruct (no counterpart in the paper, which does not
 * differentiate its filter). grad_rgb_dev: width*height float4, the loss
 * gradient with respect to each output (r, g, b); its 4th lane is ignored
 * (W is treated as a constant). Writes grad_colors_dev (3 floats per
 * frame-view record, frame order; AfrInfo.frame records) and grad_params_dev
 * (6 floats, AfrParams order; the per-block partials are added with
 * compensated FP32 sums). Gradients and
 * densities are held fixed. Weight sums are recomputed, not stored. Requires
 * a preceding afr_reconstruct on the current frame view; its params and
 * t_now are reused. Either output pointer may be NULL to skip it. */
AFR_API AfrStatus afr_reconstruct_backward(AfrContext *ctx, const float *grad_rgb_dev,
                                   float *grad_colors_dev, float *grad_params_dev,
                                   afr_stream_t stream);

/* Waits for the work issued on stream, then returns the condition recorded in
 * the context's device status word since the last call (and clears it):
 * AFR_ERR_DEVICE_CHECK for a failed device-side check (debug builds), or
 * AFR_OK. Work of this context on other streams is seen once it has
 * finished (join those streams into this one first). Only this stream is
 * synchronised, not the device. */
AFR_API AfrStatus afr_get_status(AfrContext *ctx, afr_stream_t stream);

/* Text of the most recent error on this context ("" if none). The pointer
 * stays valid until the next call on the context. */
AFR_API const char *afr_last_error(const AfrContext *ctx);

/* Synchronises the stream and fills *info. */
AFR_API AfrStatus afr_query(AfrContext *ctx, AfrInfo *info, afr_stream_t stream);

/* Number of statistics tiles. */
AFR_API AfrStatus afr_num_tiles(const AfrContext *ctx, uint32_t *n_tiles);

/* ---------------------------------------------------------------------
 * Inspection and injection (tests, checkpointing). All synchronise.
 * --------------------------------------------------------------------- */

/* Copies the deep buffer out in canonical order: for pixel p and k = 0
 * (newest) .. count-1, fields x, y, t, depth, r, g, b, mx, my as float
 * (slot_host[(p*depth + k)*9 + f], colours widened to float) and sequence
 * number seq_host[p*depth + k]. count_host gets width*height int32. Slots
 * past a pixel's count are zero. */
AFR_API AfrStatus afr_export_ring(AfrContext *ctx, int32_t *count_host, float *slot_host,
                          uint32_t *seq_host);

/* Copies the frame view out: off_host (width*height+1 uint32), and per
 * record (frame order) x', y', a^2 (a = t_now - t), r, g, b as float
 * (rec_host, 6 per record) and the sequence number. cap is the record
 * capacity of rec_host/seq_host; AFR_ERR_INVALID_ARG if the frame is larger. */
AFR_API AfrStatus afr_export_frame(AfrContext *ctx, uint32_t *off_host, float *rec_host,
                           uint32_t *seq_host, uint64_t cap);

typedef enum {
    AFR_MAP_LBAR = 0,   /* age-weighted mean luminance (NaN where empty) */
    AFR_MAP_GX = 1, AFR_MAP_GY = 2, AFR_MAP_GT = 3,
    AFR_MAP_SIGMA_S = 4, AFR_MAP_SIGMA_T = 5,
    AFR_MAP_FOOTPRINT = 6,  /* footprint radius r of the last adaptive reconstruction (export only) */
    AFR_MAP_COVERAGE = 7    /* samples in each pixel's footprint in that reconstruction (export only) */
} AfrMap;

/* Copies one width*height float map out / in. Importing a gradient map
 * replaces the estimate (the next afr_reconstruct computes widths from it);
 * importing a width map makes the next afr_reconstruct use it as is
 * (AFR_RECON_KEEP_SIGMA). */
AFR_API AfrStatus afr_export_map(AfrContext *ctx, AfrMap which, float *map_host);
AFR_API AfrStatus afr_import_map(AfrContext *ctx, AfrMap which, const float *map_host);

/* Replaces the colours of the frame view (3 floats per record, frame
 * order, device memory), e.g. to differentiate with respect to them. */
AFR_API AfrStatus afr_set_frame_colors(AfrContext *ctx, const float *rgb_dev, afr_stream_t stream);

enum { AFR_RECON_KEEP_SIGMA = 1, AFR_RECON_ADAPTIVE_SUPPORT = 2, AFR_RECON_COVERAGE_RESET = 4 };
/* afr_reconstruct with flags. AFR_RECON_KEEP_SIGMA filters with the width
 * map already in the context (imported or from the previous call).
 *
 * AFR_RECON_ADAPTIVE_SUPPORT (section 6.2, the coverage map, in gather
 * form): each pixel gets its own footprint, the integer disc of radius
 * floor(r + 1/2), where r is the mean of the radii used in the previous
 * adaptive reconstruction over the pixel's 3x3 neighbourhood, times 4 if
 * fewer than 4 samples reached the pixel then, times 0.7 if more than 32 did,
 * clamped to [0.5, 8] (single precision, one rounding per operation). The
 * radii and counts persist in the context between calls; they start as
 * r = the configured radius and "no count" (factor 1), and
 * AFR_RECON_COVERAGE_RESET returns them to that state before the update.
 * afr_reconstruct_backward and the batched form use the configured radius
 * only: backward after an adaptive reconstruction returns AFR_ERR_BAD_STATE. */
AFR_API AfrStatus afr_reconstruct_ex(AfrContext *ctx, float t_now, const AfrParams *params,
                             uint32_t flags, float *out_rgbw_dev, afr_stream_t stream);

/* Filter tuning of a context: footprint radius R (0..8; it changes results:
 * the footprint is the integer disc of radius R) and the filter's CTA tile,
 * (2*tile_bx) x (64/tile_bx) pixels with tile_bx in {2, 4, 8, 16} (default 4;
 * it does not change results). */
AFR_API AfrStatus afr_set_tuning(AfrContext *ctx, int32_t radius, int32_t tile_bx);

/* Kernel timing of the filter (instrumentation; the paper has no
 * counterpart). While enabled, each afr_reconstruct / afr_reconstruct_ex
 * records a pair of CUDA events on its stream around the filter kernel (the
 * widths kernel before it is outside the pair), for up to
 * AFR_PROFILE_MAX_LAUNCHES launches; later launches are not recorded.
 * afr_profile_filter(ctx, 1) starts a new record (the context creates its
 * events on first use), afr_profile_filter(ctx, 0) stops recording.
 * afr_profile_read waits for the recorded events, writes up to cap launch
 * durations in milliseconds to ms_host (host memory) in launch order, the
 * number recorded to *count, and clears the record. Returns
 * AFR_ERR_BAD_STATE if a stream was being captured into a CUDA graph when a
 * pair would have been recorded (such a launch is not recorded). */
enum { AFR_PROFILE_MAX_LAUNCHES = 256 };

/* Measured FP32 issue rates of the current device, the denominators of the
 * filter's roofline (instrumentation; the paper has no counterpart): every
 * thread of a grid that fills the GPU runs independent chains of one
 * operation. out_host (4 floats, host memory) receives the scalar FMA rate
 * and the paired FMA (fma.rn.f32x2) rate in TFLOP/s (2 and 4 FLOP an
 * instruction), the ex2.approx rate in Tops/s, and the SM count.
 * Synchronises the device; AFR_ERR_CUDA if a kernel fails. */
AFR_API AfrStatus afr_measure_alu_peaks(float *out_host);
AFR_API AfrStatus afr_profile_filter(AfrContext *ctx, int32_t enable);
AFR_API AfrStatus afr_profile_read(AfrContext *ctx, float *ms_host, int32_t cap, int32_t *count);

/* ---------------------------------------------------------------------
 * Batched form: many independent viewer streams (contexts) reconstructed in
 * one persistent launch (no counterpart in the paper, which renders one
 * stream). All contexts must share the colour type; at most 64.
 * --------------------------------------------------------------------- */
typedef struct AfrBatch AfrBatch;

/* Freezes the set of contexts and their filter tile shapes (largest images
 * are scheduled first). The contexts must outlive the batch. */
AFR_API AfrStatus afr_batch_create(AfrContext *const *ctxs, int32_t n, AfrBatch **out);
AFR_API void afr_batch_destroy(AfrBatch *batch);

/* afr_reconstruct for every context of the batch in one call. Contexts of
 * up to 131,072 pixels share two launches: one kernel computes the widths of
 * all their pixels, then one persistent kernel takes tiles of any of them
 * from a work queue (one atomic counter) and filters them; tiles never wait
 * for one another. Larger contexts, which fill the GPU on their own, get
 * afr_reconstruct's own launches within the call. Results equal
 * afr_reconstruct's bit for bit. outs_dev[i] receives context i's image (as
 * afr_reconstruct). Each context needs afr_estimate_gradients and
 * afr_reproject for t_now. The parameters and output pointers are staged in
 * pinned host memory owned by the batch, so the call can be captured in a
 * CUDA graph and replayed. */
AFR_API AfrStatus afr_batch_reconstruct(AfrBatch *batch, float t_now, const AfrParams *params,
                                        float *const *outs_dev, afr_stream_t stream);

/* The whole refresh of every context of the batch in one call: for each,
 * afr_estimate_gradients, afr_reproject and afr_reconstruct at t_now with
 * params, its image to outs_dev[i]. The contexts are spread over the batch's
 * own worker streams (fixed at afr_batch_create: four, each context on the
 * one with the least buffered work so far, largest contexts first), which
 * wait for the work issued on stream before the call and which stream waits
 * for after it, so independent contexts run concurrently and the call can be
 * captured in a CUDA graph. Results equal the calls in series bit for bit.
 * Reads each context's sample buffers: the same ordering rules as the calls
 * it stands for. */
AFR_API AfrStatus afr_batch_refresh(AfrBatch *batch, float t_now, const AfrParams *params,
                                    float *const *outs_dev, afr_stream_t stream);

/* ---------------------------------------------------------------------
 * Allocation-free variant (no counterpart in the paper).
 * --------------------------------------------------------------------- */

/* afr_reproject's move and binning applied directly to a caller-held batch,
 * for callers that cannot allocate device memory when they need the step
 * (a render thread with a fixed memory budget, a host whose frame callback
 * forbids allocation): it needs no context and calls no allocator. Each
 * sample of the batch that afr_insert_samples would accept is moved to
 * t_now as afr_reproject moves it and binned at the pixel holding x'; the
 * result is the frame view that afr_reproject builds from a context whose
 * queues hold the whole batch.
 *   batch        as for afr_insert_samples, colours in color_type
 *   off_dev      width*height+1 uint32: record offset of each pixel's bin
 *   rec_dev      n x float4 (x', y', a^2, bin column as int32 bits)
 *   col_dev      n colours in color_type (16 or 8 bytes each)
 *   seq_dev      n uint32: batch index of each record; within a bin of up to
 *                4096 records, records are ordered by batch index; a larger
 *                bin holds its records in an unspecified order (as
 *                afr_reproject keeps such bins in arrival order)
 *   n_frame_dev  1 uint32: number of records written (may be NULL)
 * The only scratch is one fixed device array of about 4 MB built into the
 * library, held by every GPU that loads it until the process exits; it
 * bounds width*height to 1,048,576 pixels, and n is bounded by 2^26. Larger
 * sizes return AFR_ERR_INVALID_ARG, like null or misaligned pointers. The
 * array's device address is looked up on the first call made with each
 * device current (make that call before any stream capture) and cached, so
 * calls made after a cudaDeviceReset are undefined. All calls
 * share the array, so calls that overlap on the GPU race and must be
 * serialised by the caller. Asynchronous on the stream. */
AFR_API AfrStatus afr_reproject_batch_static(const AfrSampleBatch *batch, uint32_t n, int32_t width,
                                             int32_t height, int32_t color_type, float t_now, uint32_t *off_dev,
                                             float *rec_dev, void *col_dev, uint32_t *seq_dev,
                                             uint32_t *n_frame_dev, afr_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif

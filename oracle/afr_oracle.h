/*
 * afr_oracle.h -- CPU oracle of the adaptive frameless reconstruction path.
 *
 * TEST INFRASTRUCTURE. This is a plain, slow, step-by-step restatement of the
 * reconstruction method of Dayal, Woolley, Watson and Luebke, "Adaptive
 * Frameless Rendering" (sections 4, 4.1, 5.1, 5.2, 6.1, 6.2), written for
 * checking the CUDA library, never for producing results. Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg call it. It shares no code,
 * header, table or helper with the CUDA library.
 *
 * Arithmetic is double precision, except the reprojected position, whose
 * floor decides the destination bin: it is taken in single precision with one
 * rounding per operation (no contraction), as the CUDA path takes it.
 *
 * Ring layout (canonical, used for comparisons): for pixel p = y*W + x and
 * slot k (0 = newest), field f of the sample is slot[((size_t)p*b + k)*AFO_NF + f]
 * and its insertion sequence number is seq[(size_t)p*b + k].
 */
#ifndef AFR_ORACLE_H
#define AFR_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Threads of the loops over independent pixels, rows and tiles (OpenMP
 * builds; results do not depend on the count). */
void afo_set_threads(int n);
int afo_max_threads(void);

enum { AFO_X = 0, AFO_Y, AFO_T, AFO_DEPTH, AFO_R, AFO_G, AFO_B, AFO_MX, AFO_MY, AFO_NF };
/* reprojected (frame-view) record: x', y', t, r, g, b */
enum { AFO_RX = 0, AFO_RY, AFO_RT, AFO_RR, AFO_RG, AFO_RB, AFO_NR };
/* tile statistics record */
enum { AFO_TN = 0, AFO_TEMPTY, AFO_TMEANL, AFO_TVARL, AFO_TGX, AFO_TGY, AFO_TGT, AFO_TU, AFO_NT };
/* filter parameters theta */
enum { AFO_ALPHA_S = 0, AFO_BETA_S, AFO_CLAMP_S, AFO_ALPHA_T, AFO_BETA_T, AFO_CLAMP_T, AFO_NP };

/* Section 6.2 with camera matrices: every resident sample's 3D hit point
 * (world_by_seq[4*seq .. 4*seq+2], looked up by its sequence number) is
 * projected with the row-major 4x4 matrix vp: c = vp (X, Y, Z, 1), each row
 * summed left to right; x' = (c_x / c_w * 1/2 + 1/2) W + m_x a and
 * y' = (c_y / c_w * 1/2 + 1/2) H + m_y a with a = t_now - t, single
 * precision, one rounding per operation. Samples with c_w <= 0 or leaving
 * the image are dropped. Frame view as afo_reproject. */
int64_t afo_reproject_camera(int W, int H, int b, const int32_t *count, const float *slot,
                             const uint32_t *seq, const float *world_by_seq, const float *vp,
                             float t_now, uint32_t *off, float *rec, uint32_t *rseq, int64_t cap,
                             int64_t *dropped);

/* Section 5.2: the reconstructor's own deep buffer, one temporally ordered
 * queue of the N most recent samples over the whole image. Accepted samples
 * (as afo_ingest accepts them) of the batch enter in index order at slot
 * (*total mod N); *total counts the accepted samples so far. Returns the
 * number rejected. q holds N*AFO_NF floats, qseq N sequence numbers. */
int64_t afo_fifo_insert(int W, int H, int64_t N, int64_t *total, float *q, uint32_t *qseq,
                        uint32_t seq0, int64_t n, const float *pos, const float *col,
                        const float *mo);

/* Section 4: push a batch into the per-pixel deep-buffer queues. Returns the
 * number of rejected samples. seq of sample i is seq0 + i. */
int64_t afo_ingest(int W, int H, int b, int32_t *count, float *slot, uint32_t *seq,
                   uint32_t seq0, int64_t n, const float *pos, const float *col,
                   const float *mo);

/* Sections 4 and 4.1: per-pixel age-weighted mean luminance and gradients.
 * Lbar is NaN for an empty pixel. */
void afo_gradients(int W, int H, int b, const int32_t *count, const float *slot,
                   const uint32_t *seq, float t_now, double *Lbar, double *Gx,
                   double *Gy, double *Gt);

/* Sections 4, 4.2 and 6.1: per-tile statistics (AFO_NT doubles per tile,
 * tiles in row-major order of a ceil(H/S)-by-ceil(W/S) grid). */
void afo_tile_feedback(int W, int H, int b, int S, const int32_t *count,
                       const float *slot, float t_now, const double *Gx,
                       const double *Gy, const double *Gt, double m, double *out);

/* Section 6.2: reproject every resident sample to t_now and bin it into a
 * CSR frame view (bins row-major, within a bin by seq ascending). off has P+1
 * entries, rec has cap*AFO_NR floats. Returns the number of binned samples
 * (or -1 if cap is too small); *dropped gets the off-image count. */
int64_t afo_reproject(int W, int H, int b, const int32_t *count, const float *slot,
                      const uint32_t *seq, float t_now, uint32_t *off, float *rec,
                      uint32_t *rseq, int64_t cap, int64_t *dropped);

/* Section 5.1: filter widths from density and gradients (tile size S). */
void afo_sigma(int W, int H, int b, int S, const int32_t *count, const double *Gx,
               const double *Gy, const double *Gt, const double *theta,
               double window, double eps, double *sig_s, double *sig_t);

/* Sections 5.1 and 5.2: normalised space-time Gaussian gather over the
 * integer disc of radius R. out has 4 doubles per pixel (r, g, b, W). If
 * pixels != NULL only those n_pixels pixel indices are filtered (others left
 * untouched). */
void afo_filter(int W, int H, int R, const uint32_t *off, const float *rec,
                float t_now, const double *sig_s, const double *sig_t,
                const int64_t *pixels, int64_t n_pixels, double *out);

/* The same sum written over all samples for every pixel, with no bins. */
void afo_filter_brute(int W, int H, int R, int64_t n, const float *rec, float t_now,
                      const double *sig_s, const double *sig_t, double *out);

/* Sections 6.1 and 4.1: tile error and gain control from the records of
 * afo_tile_feedback (AFO_NT doubles per tile). occluded: occluded samples per
 * tile (NULL: none). E[t] = s_t (kappa v_t / sum v + lambda u_t / sum u +
 * (1 - kappa - lambda) o_t / sum o) with s_t the tile's pixel count and
 * o_t = occluded_t / (s_t b); a term whose sum over tiles is 0 adds 0.
 * gain[5] = (dC/ds, dC/dt, T, S*, N*): the image means over non-empty pixels
 * of (G_x + G_y) / 2 and of G_t, the mean over tiles holding samples of their
 * mean sample age max(0, t_now - t), the tile width S* = importance dC/dt T /
 * max(dC/ds, eps) that balances the two, and the tile count W H / S*^2
 * clamped to [1, W H]. */
void afo_tile_error(int W, int H, int b, int S, const int32_t *count, const float *slot,
                    float t_now, const double *tiles, const double *occluded, double kappa,
                    double lambda, double importance, double eps, double *E, double *gain);

/* Section 6.2, coverage map, in gather form: the footprint radius of each
 * pixel for the next image is the mean of the radii used for the previous
 * image over the pixel's 3x3 neighbourhood (clipped at the border), times 4
 * where fewer than 4 samples reached the pixel, times 0.7 where more than 32
 * did (n_prev < 0: no information, times 1), clamped to [r_min, r_max]; the
 * integer disc radius is floor(r + 1/2). Single precision, one rounding per
 * operation: the result decides an integer. */
void afo_coverage_update(int W, int H, const float *r_prev, const int32_t *n_prev,
                         float r_min, float r_max, float *r_next, int32_t *R_next);

/* Number of frame-view records in each pixel's integer disc of radius Rp[p]. */
void afo_coverage_count(int W, int H, const int32_t *Rp, const uint32_t *off, int32_t *n);

/* afo_filter and afo_filter_brute with a per-pixel disc radius Rp. */
void afo_filter_var(int W, int H, const int32_t *Rp, const uint32_t *off, const float *rec,
                    float t_now, const double *sig_s, const double *sig_t,
                    const int64_t *pixels, int64_t n_pixels, double *out);
void afo_filter_brute_var(int W, int H, const int32_t *Rp, int64_t n, const float *rec,
                          float t_now, const double *sig_s, const double *sig_t, double *out);

/* Adjoint of the filter and the width mapping for a loss with per-pixel
 * gradient grad_rgb (3 doubles per pixel): gradient with respect to the
 * colours of the frame-view records (3 doubles per record) and to theta. */
void afo_backward(int W, int H, int b, int S, int R, const int32_t *count,
                  const double *Gx, const double *Gy, const double *Gt,
                  const double *theta, double window, double eps,
                  const uint32_t *off, const float *rec, float t_now,
                  const double *grad_rgb, double *grad_col, double *grad_theta);

#ifdef __cplusplus
}
#endif
#endif

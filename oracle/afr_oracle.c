/*
 * afr_oracle.c -- CPU oracle of the adaptive frameless reconstruction path.
 *
 * TEST INFRASTRUCTURE: see afr_oracle.h. Each function restates one step of
 * Dayal, Woolley, Watson and Luebke, "Adaptive Frameless Rendering", in the
 * paper's order and notation, with plain loops and no blocking or fusion.
 * Build with -ffp-contract=off so that the single-precision reprojection is
 * evaluated with one rounding per operation.
 */
#include "afr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads for the loops over independent pixels, rows and tiles. Each
 * pixel's (tile's, bin's) computation and every floating-point sum keep
 * their order, so results do not depend on the thread count. */
void afo_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int afo_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

static int thread_count(void)
{
#ifdef _OPENMP
    return omp_get_num_threads();
#else
    return 1;
#endif
}

static int thread_index(void)
{
#ifdef _OPENMP
    return omp_get_thread_num();
#else
    return 0;
#endif
}

/* Luminance of an RGB colour. The paper measures colour change as luminance
 * change (sections 4, 4.1) without naming the weights; Rec. 709 weights are
 * used. */
static double luminance(double r, double g, double b)
{
    return 0.2126 * r + 0.7152 * g + 0.0722 * b;
}

/* Section 4: sample weights fall off as exp(-3.47 a) with age a, so a sample
 * one window old counts about 1/32. Samples from the future count fully. */
static double age_weight(double t_now, double t)
{
    double a = t_now - t;
    if (a < 0.0) a = 0.0;
    return exp(-3.47 * a);
}

static const float *sample_at(const float *slot, int b, size_t p, int k)
{
    return slot + ((size_t)p * b + k) * AFO_NF;
}

/* ------------------------------------------------------------------------ */
/* Section 4: each pixel of the deep buffer is a queue of depth b. A new sample
 * enters at the front; when the queue is full the sample at the back leaves. */
int64_t afo_ingest(int W, int H, int b, int32_t *count, float *slot, uint32_t *seq,
                   uint32_t seq0, int64_t n, const float *pos, const float *col,
                   const float *mo)
{
    int64_t rejected = 0;
    /* Every pixel's queue is independent of the others, so each thread takes
     * a band of rows and pushes, in input order, the samples that fall in it. */
#pragma omp parallel reduction(+ : rejected)
    {
        const int nt = thread_count(), me = thread_index();
        const int y0 = (int)((int64_t)H * me / nt), y1 = (int)((int64_t)H * (me + 1) / nt);
        for (int64_t i = 0; i < n; ++i) {
            const float *ps = pos + 4 * i, *cs = col + 4 * i, *ms = mo + 2 * i;
            float x = ps[0], y = ps[1], t = ps[2];
            int ok = isfinite(x) && isfinite(y) && isfinite(t) && isfinite(cs[0]) &&
                     isfinite(cs[1]) && isfinite(cs[2]) && isfinite(ms[0]) && isfinite(ms[1]);
            if (!ok || x < 0.0f || y < 0.0f || x >= (float)W || y >= (float)H) {
                if (me == 0) ++rejected;
                continue;
            }
            int row = (int)floorf(y);
            if (row < y0 || row >= y1) continue;
            size_t p = (size_t)row * (size_t)W + (size_t)(int)floorf(x);
            int c = count[p];
            int last = c < b ? c : b - 1;
            for (int k = last; k > 0; --k) {
                memcpy(slot + ((size_t)p * b + k) * AFO_NF, slot + ((size_t)p * b + k - 1) * AFO_NF,
                       AFO_NF * sizeof(float));
                seq[(size_t)p * b + k] = seq[(size_t)p * b + k - 1];
            }
            float *s = slot + (size_t)p * b * AFO_NF;
            s[AFO_X] = x;
            s[AFO_Y] = y;
            s[AFO_T] = t;
            s[AFO_DEPTH] = ps[3];
            s[AFO_R] = cs[0];
            s[AFO_G] = cs[1];
            s[AFO_B] = cs[2];
            s[AFO_MX] = ms[0];
            s[AFO_MY] = ms[1];
            seq[(size_t)p * b] = seq0 + (uint32_t)i;
            if (c < b) count[p] = c + 1;
        }
    }
    return rejected;
}

/* ------------------------------------------------------------------------ */
/* Section 5.2: the reconstructor stores the N most recent samples of the
 * whole image in one queue ordered by time of arrival; a new sample replaces
 * the oldest once the queue is full. */
int64_t afo_fifo_insert(int W, int H, int64_t N, int64_t *total, float *q, uint32_t *qseq,
                        uint32_t seq0, int64_t n, const float *pos, const float *col,
                        const float *mo)
{
    int64_t rejected = 0;
    for (int64_t i = 0; i < n; ++i) {
        const float *ps = pos + 4 * i, *cs = col + 4 * i, *ms = mo + 2 * i;
        float x = ps[0], y = ps[1], t = ps[2];
        int ok = isfinite(x) && isfinite(y) && isfinite(t) && isfinite(cs[0]) &&
                 isfinite(cs[1]) && isfinite(cs[2]) && isfinite(ms[0]) && isfinite(ms[1]);
        if (!ok || x < 0.0f || y < 0.0f || x >= (float)W || y >= (float)H) {
            ++rejected;
            continue;
        }
        int64_t k = *total % N;
        float *s = q + (size_t)k * AFO_NF;
        s[AFO_X] = x;
        s[AFO_Y] = y;
        s[AFO_T] = t;
        s[AFO_DEPTH] = ps[3];
        s[AFO_R] = cs[0];
        s[AFO_G] = cs[1];
        s[AFO_B] = cs[2];
        s[AFO_MX] = ms[0];
        s[AFO_MY] = ms[1];
        qseq[k] = seq0 + (uint32_t)i;
        *total += 1;
    }
    return rejected;
}

/* ------------------------------------------------------------------------ */
/* Sections 4 and 4.1. The pixel's luminance is the age-weighted mean of its
 * queue. The spatial gradient in x is the mean of the one-sided absolute
 * luminance differences to the left and right neighbours (those that exist
 * and hold samples); likewise in y. The temporal gradient compares samples
 * at the same pixel made at different times: with the queue ordered newest
 * first by time, it is the age-weighted sum of |dL| over consecutive samples
 * divided by the age-weighted sum of their time differences, each pair
 * weighted by the age of its newer sample. */
void afo_gradients(int W, int H, int b, const int32_t *count, const float *slot,
                   const uint32_t *seq, float t_now, double *Lbar, double *Gx,
                   double *Gy, double *Gt)
{
    const int64_t P = (int64_t)W * H;
#pragma omp parallel
    {
    int *order = (int *)malloc(sizeof(int) * (size_t)(b > 0 ? b : 1));
#pragma omp for schedule(static)
    for (int64_t p = 0; p < P; ++p) {
        int n = count[p];
        if (n == 0) {
            Lbar[p] = NAN;
            Gt[p] = 0.0;
            continue;
        }
        double sw = 0.0, swl = 0.0;
        for (int k = 0; k < n; ++k) {
            const float *s = sample_at(slot, b, p, k);
            double w = age_weight(t_now, s[AFO_T]);
            sw += w;
            swl += w * luminance(s[AFO_R], s[AFO_G], s[AFO_B]);
        }
        Lbar[p] = swl / sw;

        /* newest first by time; equal times by sequence number, newest first */
        for (int k = 0; k < n; ++k) order[k] = k;
        for (int k = 1; k < n; ++k) {
            int v = order[k], j = k - 1;
            float tv = sample_at(slot, b, p, v)[AFO_T];
            uint32_t sv = seq[p * b + v];
            while (j >= 0) {
                float tj = sample_at(slot, b, p, order[j])[AFO_T];
                uint32_t sj = seq[p * b + order[j]];
                if (tj > tv || (tj == tv && sj > sv)) break;
                order[j + 1] = order[j];
                --j;
            }
            order[j + 1] = v;
        }
        double num = 0.0, den = 0.0;
        for (int k = 0; k + 1 < n; ++k) {
            const float *s0 = sample_at(slot, b, p, order[k]);
            const float *s1 = sample_at(slot, b, p, order[k + 1]);
            double w = age_weight(t_now, s0[AFO_T]);
            double L0 = luminance(s0[AFO_R], s0[AFO_G], s0[AFO_B]);
            double L1 = luminance(s1[AFO_R], s1[AFO_G], s1[AFO_B]);
            num += w * fabs(L0 - L1);
            den += w * ((double)s0[AFO_T] - (double)s1[AFO_T]);
        }
        Gt[p] = (n >= 2 && den > 0.0) ? num / den : 0.0;
    }
    free(order);
    }

#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            if (count[p] == 0) {
                Gx[p] = 0.0;
                Gy[p] = 0.0;
                continue;
            }
            double sum = 0.0;
            int m = 0;
            if (x > 0 && count[p - 1] > 0) { sum += fabs(Lbar[p] - Lbar[p - 1]); ++m; }
            if (x + 1 < W && count[p + 1] > 0) { sum += fabs(Lbar[p] - Lbar[p + 1]); ++m; }
            Gx[p] = m ? sum / m : 0.0;
            sum = 0.0;
            m = 0;
            if (y > 0 && count[p - W] > 0) { sum += fabs(Lbar[p] - Lbar[p - W]); ++m; }
            if (y + 1 < H && count[p + W] > 0) { sum += fabs(Lbar[p] - Lbar[p + W]); ++m; }
            Gy[p] = m ? sum / m : 0.0;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Sections 4, 4.2 and 6.1, over fixed S-by-S tiles: sample count, age-weighted
 * mean and variance of luminance over the tile's block, mean gradients over
 * its non-empty pixels, empty buffer slots, and the undersampling measure
 * u = 1 - min(1, m * mean_empty / empty), with mean_empty the mean number of
 * empty slots per tile and u = 0 for a tile with no empty slot. */
void afo_tile_feedback(int W, int H, int b, int S, const int32_t *count,
                       const float *slot, float t_now, const double *Gx,
                       const double *Gy, const double *Gt, double m, double *out)
{
    int ntx = (W + S - 1) / S, nty = (H + S - 1) / S;
    double empty_sum = 0.0;
#pragma omp parallel for collapse(2) schedule(static)
    for (int ty = 0; ty < nty; ++ty) {
        for (int tx = 0; tx < ntx; ++tx) {
            int x0 = tx * S, y0 = ty * S;
            int x1 = x0 + S < W ? x0 + S : W, y1 = y0 + S < H ? y0 + S : H;
            double n = 0.0, sw = 0.0, swl = 0.0, gx = 0.0, gy = 0.0, gt = 0.0, nonempty = 0.0;
            for (int y = y0; y < y1; ++y) {
                for (int x = x0; x < x1; ++x) {
                    size_t p = (size_t)y * W + x;
                    n += count[p];
                    for (int k = 0; k < count[p]; ++k) {
                        const float *s = sample_at(slot, b, p, k);
                        double w = age_weight(t_now, s[AFO_T]);
                        sw += w;
                        swl += w * luminance(s[AFO_R], s[AFO_G], s[AFO_B]);
                    }
                    if (count[p] > 0) {
                        gx += Gx[p];
                        gy += Gy[p];
                        gt += Gt[p];
                        nonempty += 1.0;
                    }
                }
            }
            double mean = sw > 0.0 ? swl / sw : 0.0, sq = 0.0;
            for (int y = y0; y < y1; ++y) {
                for (int x = x0; x < x1; ++x) {
                    size_t p = (size_t)y * W + x;
                    for (int k = 0; k < count[p]; ++k) {
                        const float *s = sample_at(slot, b, p, k);
                        double d = luminance(s[AFO_R], s[AFO_G], s[AFO_B]) - mean;
                        sq += age_weight(t_now, s[AFO_T]) * d * d;
                    }
                }
            }
            double *o = out + ((size_t)ty * ntx + tx) * AFO_NT;
            o[AFO_TN] = n;
            o[AFO_TEMPTY] = (double)(x1 - x0) * (y1 - y0) * b - n;
            o[AFO_TMEANL] = mean;
            o[AFO_TVARL] = sw > 0.0 ? sq / sw : 0.0;
            o[AFO_TGX] = nonempty > 0.0 ? gx / nonempty : 0.0;
            o[AFO_TGY] = nonempty > 0.0 ? gy / nonempty : 0.0;
            o[AFO_TGT] = nonempty > 0.0 ? gt / nonempty : 0.0;
        }
    }
    for (int i = 0; i < ntx * nty; ++i) empty_sum += out[(size_t)i * AFO_NT + AFO_TEMPTY];
    double mean_empty = empty_sum / ((double)ntx * nty);
    for (int i = 0; i < ntx * nty; ++i) {
        double *o = out + (size_t)i * AFO_NT;
        double e = o[AFO_TEMPTY];
        double r = e > 0.0 ? m * mean_empty / e : 0.0;
        o[AFO_TU] = e > 0.0 ? 1.0 - (r < 1.0 ? r : 1.0) : 0.0;
    }
}

/* ------------------------------------------------------------------------ */
/* Section 6.2: every resident sample moves along its screen-space velocity to
 * the display time, x' = x + m_x (t_now - t), and is binned at the pixel that
 * contains x'. Samples that leave the image are dropped. */
typedef struct {
    uint32_t bin, seq;
    float v[AFO_NR];
} ReprojEntry;

static int entry_cmp(const void *a, const void *b)
{
    const ReprojEntry *ea = (const ReprojEntry *)a, *eb = (const ReprojEntry *)b;
    if (ea->bin != eb->bin) return ea->bin < eb->bin ? -1 : 1;
    if (ea->seq != eb->seq) return ea->seq < eb->seq ? -1 : 1;
    return 0;
}

int64_t afo_reproject(int W, int H, int b, const int32_t *count, const float *slot,
                      const uint32_t *seq, float t_now, uint32_t *off, float *rec,
                      uint32_t *rseq, int64_t cap, int64_t *dropped)
{
    size_t P = (size_t)W * H;
    int nbands = afo_max_threads();
    if (nbands > H) nbands = H;
    if (nbands < 1) nbands = 1;
    ReprojEntry **band = (ReprojEntry **)calloc((size_t)nbands, sizeof(ReprojEntry *));
    size_t *bn = (size_t *)calloc((size_t)nbands, sizeof(size_t));
    int64_t drop = 0;
    /* Band k collects the samples whose destination row lies in its rows and
     * sorts them by (bin, sequence number); bins are row-major, so the bands
     * in order are the whole frame view in that order. */
#pragma omp parallel for schedule(static, 1) reduction(+ : drop)
    for (int k = 0; k < nbands; ++k) {
        const int y0 = (int)((int64_t)H * k / nbands), y1 = (int)((int64_t)H * (k + 1) / nbands);
        ReprojEntry *e = NULL;
        size_t n = 0;
        for (int pass = 0; pass < 2; ++pass) {   /* count the band's samples, then store them */
            if (pass == 1) {
                e = (ReprojEntry *)malloc(sizeof(ReprojEntry) * (n ? n : 1));
                n = 0;
            }
        for (size_t p = 0; p < P; ++p) {
            for (int j = 0; j < count[p]; ++j) {
                const float *s = sample_at(slot, b, p, j);
                float a = t_now - s[AFO_T];
                float dx = s[AFO_MX] * a;
                float dy = s[AFO_MY] * a;
                float xp = s[AFO_X] + dx;
                float yp = s[AFO_Y] + dy;
                if (!(xp >= 0.0f && xp < (float)W && yp >= 0.0f && yp < (float)H)) {
                    if (k == 0 && pass == 1) ++drop;
                    continue;
                }
                int row = (int)floorf(yp);
                if (row < y0 || row >= y1) continue;
                if (pass == 0) {
                    ++n;
                    continue;
                }
                e[n].bin = (uint32_t)(row * W + (int)floorf(xp));
                e[n].seq = seq[p * b + j];
                e[n].v[AFO_RX] = xp;
                e[n].v[AFO_RY] = yp;
                e[n].v[AFO_RT] = s[AFO_T];
                e[n].v[AFO_RR] = s[AFO_R];
                e[n].v[AFO_RG] = s[AFO_G];
                e[n].v[AFO_RB] = s[AFO_B];
                ++n;
            }
        }
        }
        qsort(e, n, sizeof(ReprojEntry), entry_cmp);
        band[k] = e;
        bn[k] = n;
    }
    size_t n = 0;
    for (int k = 0; k < nbands; ++k) n += bn[k];
    if (dropped) *dropped = drop;
    if ((int64_t)n > cap) {
        for (int k = 0; k < nbands; ++k) free(band[k]);
        free(band);
        free(bn);
        return -1;
    }
    for (size_t q = 0; q <= P; ++q) off[q] = 0;
    size_t i = 0;
    for (int k = 0; k < nbands; ++k) {
        for (size_t j = 0; j < bn[k]; ++j, ++i) {
            const ReprojEntry *e = band[k] + j;
            off[e->bin + 1] += 1;
            memcpy(rec + i * AFO_NR, e->v, sizeof(float) * AFO_NR);
            rseq[i] = e->seq;
        }
        free(band[k]);
    }
    for (size_t q = 0; q < P; ++q) off[q + 1] += off[q];
    free(band);
    free(bn);
    return (int64_t)n;
}

/* Section 6.2: the reconstructor reprojects by rendering the stored hit points
 * with the current camera; a sample's own motion (if any) is added on screen. */
static int project(const float *vp, const float *w, int W, int H, float *sx, float *sy)
{
    float cx = vp[0] * w[0];
    cx = cx + vp[1] * w[1];
    cx = cx + vp[2] * w[2];
    cx = cx + vp[3];
    float cy = vp[4] * w[0];
    cy = cy + vp[5] * w[1];
    cy = cy + vp[6] * w[2];
    cy = cy + vp[7];
    float cw = vp[12] * w[0];
    cw = cw + vp[13] * w[1];
    cw = cw + vp[14] * w[2];
    cw = cw + vp[15];
    if (!(cw > 0.0f)) return 0;
    float nx = cx / cw, ny = cy / cw;
    *sx = (nx * 0.5f + 0.5f) * (float)W;
    *sy = (ny * 0.5f + 0.5f) * (float)H;
    return 1;
}

int64_t afo_reproject_camera(int W, int H, int b, const int32_t *count, const float *slot,
                             const uint32_t *seq, const float *world_by_seq, const float *vp,
                             float t_now, uint32_t *off, float *rec, uint32_t *rseq, int64_t cap,
                             int64_t *dropped)
{
    size_t P = (size_t)W * H, total = 0;
    for (size_t p = 0; p < P; ++p) total += (size_t)count[p];
    ReprojEntry *e = (ReprojEntry *)malloc(sizeof(ReprojEntry) * (total ? total : 1));
    size_t n = 0;
    int64_t drop = 0;
    for (size_t p = 0; p < P; ++p) {
        for (int k = 0; k < count[p]; ++k) {
            const float *s = sample_at(slot, b, p, k);
            uint32_t sq = seq[p * b + k];
            float sx, sy;
            int front = project(vp, world_by_seq + (size_t)sq * 4, W, H, &sx, &sy);
            float a = t_now - s[AFO_T];
            float xp = sx + s[AFO_MX] * a;
            float yp = sy + s[AFO_MY] * a;
            if (!front || !(xp >= 0.0f && xp < (float)W && yp >= 0.0f && yp < (float)H)) {
                ++drop;
                continue;
            }
            e[n].bin = (uint32_t)((int)floorf(yp) * W + (int)floorf(xp));
            e[n].seq = sq;
            e[n].v[AFO_RX] = xp;
            e[n].v[AFO_RY] = yp;
            e[n].v[AFO_RT] = s[AFO_T];
            e[n].v[AFO_RR] = s[AFO_R];
            e[n].v[AFO_RG] = s[AFO_G];
            e[n].v[AFO_RB] = s[AFO_B];
            ++n;
        }
    }
    if (dropped) *dropped = drop;
    if ((int64_t)n > cap) {
        free(e);
        return -1;
    }
    qsort(e, n, sizeof(ReprojEntry), entry_cmp);
    for (size_t q = 0; q <= P; ++q) off[q] = 0;
    for (size_t i = 0; i < n; ++i) off[e[i].bin + 1] += 1;
    for (size_t q = 0; q < P; ++q) off[q + 1] += off[q];
    for (size_t i = 0; i < n; ++i) {
        memcpy(rec + i * AFO_NR, e[i].v, sizeof(float) * AFO_NR);
        rseq[i] = e[i].seq;
    }
    free(e);
    return (int64_t)n;
}

/* ------------------------------------------------------------------------ */
/* Section 5.1. The local sampling rate R_l (samples per pixel per window) is
 * read from the sampler's tiling, here the fixed tile holding the pixel, and
 * V_S = 1 / R_l. The extents satisfy e_x G_x = e_y G_y = e_t G_t with
 * e_x e_y e_t = V_S. With one spatial extent e_s for both axes and the mean
 * spatial gradient G_s this gives e_s = cbrt(V_S G_t / G_s) and
 * e_t = cbrt(V_S G_s^2 / G_t^2). The Gaussian widths are the extents mapped by
 * a scale, an offset and an upper clamp per axis, with fixed lower bounds. */
static void tile_counts(int W, int H, int S, const int32_t *count, double *nt, double *at)
{
    int ntx = (W + S - 1) / S, nty = (H + S - 1) / S;
    for (int i = 0; i < ntx * nty; ++i) nt[i] = at[i] = 0.0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            int tile = (y / S) * ntx + (x / S);
            nt[tile] += count[(size_t)y * W + x];
            at[tile] += 1.0;
        }
}

typedef struct {
    double es, et, raw_s, raw_t, sig_s, sig_t;
} Widths;

static Widths widths_at(double V, double gx, double gy, double gt, const double *th,
                        double eps)
{
    Widths w;
    double Gs = 0.5 * (gx + gy);
    if (Gs < eps) Gs = eps;
    double Gtp = gt < eps ? eps : gt;
    w.es = cbrt(V * Gtp / Gs);
    w.et = cbrt(V * Gs * Gs / (Gtp * Gtp));
    w.raw_s = th[AFO_ALPHA_S] * w.es + th[AFO_BETA_S];
    w.raw_t = th[AFO_ALPHA_T] * w.et + th[AFO_BETA_T];
    double s = w.raw_s > 0.5 ? w.raw_s : 0.5;
    w.sig_s = s < th[AFO_CLAMP_S] ? s : th[AFO_CLAMP_S];
    double t = w.raw_t > 0.05 ? w.raw_t : 0.05;
    w.sig_t = t < th[AFO_CLAMP_T] ? t : th[AFO_CLAMP_T];
    return w;
}

static double volume_at(int x, int y, int W, int S, const double *nt, const double *at,
                        double window)
{
    int ntx = (W + S - 1) / S;
    int tile = (y / S) * ntx + (x / S);
    return nt[tile] > 0.0 ? at[tile] * window / nt[tile] : at[tile] * window;
}

void afo_sigma(int W, int H, int b, int S, const int32_t *count, const double *Gx,
               const double *Gy, const double *Gt, const double *theta,
               double window, double eps, double *sig_s, double *sig_t)
{
    (void)b;
    int ntiles = ((W + S - 1) / S) * ((H + S - 1) / S);
    double *nt = (double *)malloc(sizeof(double) * ntiles);
    double *at = (double *)malloc(sizeof(double) * ntiles);
    tile_counts(W, H, S, count, nt, at);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            size_t p = (size_t)y * W + x;
            Widths w = widths_at(volume_at(x, y, W, S, nt, at, window), Gx[p], Gy[p], Gt[p],
                                 theta, eps);
            sig_s[p] = w.sig_s;
            sig_t[p] = w.sig_t;
        }
    free(nt);
    free(at);
}

/* ------------------------------------------------------------------------ */
/* Sections 5.1 and 5.2: the pixel's colour is the normalised weighted average
 * of the samples near it, each weighted by a space-time Gaussian centred at
 * the pixel centre and the display time, with the pixel's own widths. The
 * footprint is the integer disc of bins within R of the pixel's bin. */
static double gauss_weight(double d2, double a, double ss, double st)
{
    return exp(-d2 / (2.0 * ss * ss) - a * a / (2.0 * st * st));
}

static void filter_pixel(int W, int H, int R, const uint32_t *off, const float *rec,
                         float t_now, double ss, double st, int i, int j, double *o)
{
    double cx = i + 0.5, cy = j + 0.5, sr = 0.0, sg = 0.0, sb = 0.0, sw = 0.0;
    for (int dj = -R; dj <= R; ++dj)
        for (int di = -R; di <= R; ++di) {
            int qi = i + di, qj = j + dj;
            if (di * di + dj * dj > R * R || qi < 0 || qj < 0 || qi >= W || qj >= H) continue;
            size_t q = (size_t)qj * W + qi;
            for (uint32_t e = off[q]; e < off[q + 1]; ++e) {
                const float *r = rec + (size_t)e * AFO_NR;
                double dx = (double)r[AFO_RX] - cx, dy = (double)r[AFO_RY] - cy;
                double a = (double)t_now - (double)r[AFO_RT];
                double w = gauss_weight(dx * dx + dy * dy, a, ss, st);
                sr += w * r[AFO_RR];
                sg += w * r[AFO_RG];
                sb += w * r[AFO_RB];
                sw += w;
            }
        }
    o[0] = sw > 0.0 ? sr / sw : 0.0;
    o[1] = sw > 0.0 ? sg / sw : 0.0;
    o[2] = sw > 0.0 ? sb / sw : 0.0;
    o[3] = sw;
}

void afo_filter(int W, int H, int R, const uint32_t *off, const float *rec,
                float t_now, const double *sig_s, const double *sig_t,
                const int64_t *pixels, int64_t n_pixels, double *out)
{
    if (pixels) {
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t k = 0; k < n_pixels; ++k) {
            int64_t p = pixels[k];
            filter_pixel(W, H, R, off, rec, t_now, sig_s[p], sig_t[p], (int)(p % W),
                         (int)(p / W), out + p * 4);
        }
        return;
    }
#pragma omp parallel for schedule(dynamic, 4)
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            size_t p = (size_t)j * W + i;
            filter_pixel(W, H, R, off, rec, t_now, sig_s[p], sig_t[p], i, j, out + p * 4);
        }
}

void afo_filter_brute(int W, int H, int R, int64_t n, const float *rec, float t_now,
                      const double *sig_s, const double *sig_t, double *out)
{
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            size_t p = (size_t)j * W + i;
            double cx = i + 0.5, cy = j + 0.5, acc[4] = {0.0, 0.0, 0.0, 0.0};
            for (int64_t e = 0; e < n; ++e) {
                const float *r = rec + (size_t)e * AFO_NR;
                int qi = (int)floorf(r[AFO_RX]), qj = (int)floorf(r[AFO_RY]);
                if ((qi - i) * (qi - i) + (qj - j) * (qj - j) > R * R) continue;
                double dx = (double)r[AFO_RX] - cx, dy = (double)r[AFO_RY] - cy;
                double a = (double)t_now - (double)r[AFO_RT];
                double w = gauss_weight(dx * dx + dy * dy, a, sig_s[p], sig_t[p]);
                acc[0] += w * r[AFO_RR];
                acc[1] += w * r[AFO_RG];
                acc[2] += w * r[AFO_RB];
                acc[3] += w;
            }
            for (int c = 0; c < 3; ++c) out[p * 4 + c] = acc[3] > 0.0 ? acc[c] / acc[3] : 0.0;
            out[p * 4 + 3] = acc[3];
        }
}

/* ------------------------------------------------------------------------ */
/* Section 6.1: a tile's error mixes its share of the colour variation, of the
 * undersampling and of the occlusion over all tiles, scaled by its size.
 * Section 4.1: the gain control balances spatial change across a tile
 * against temporal change over the samples' ages, dC/ds S = i dC/dt T. */
void afo_tile_error(int W, int H, int b, int S, const int32_t *count, const float *slot,
                    float t_now, const double *tiles, const double *occluded, double kappa,
                    double lambda, double importance, double eps, double *E, double *gain)
{
    int ntx = (W + S - 1) / S, nty = (H + S - 1) / S, nt = ntx * nty;
    double sv = 0.0, su = 0.0, so = 0.0, sgs = 0.0, sgt = 0.0, nonempty = 0.0, sage = 0.0, nage = 0.0;
    for (int t = 0; t < nt; ++t) {
        int tx = t % ntx, ty = t / ntx;
        int x0 = tx * S, y0 = ty * S;
        int x1 = x0 + S < W ? x0 + S : W, y1 = y0 + S < H ? y0 + S : H;
        double A = (double)(x1 - x0) * (y1 - y0);
        const double *r = tiles + (size_t)t * AFO_NT;
        sv += r[AFO_TVARL];
        su += r[AFO_TU];
        if (occluded) so += occluded[t] / (A * b);
        /* the tile records hold means over non-empty pixels: undo them */
        double ne = 0.0, age = 0.0;
        for (int y = y0; y < y1; ++y)
            for (int x = x0; x < x1; ++x) {
                size_t p = (size_t)y * W + x;
                if (count[p] > 0) ne += 1.0;
                for (int k = 0; k < count[p]; ++k) {
                    double a = (double)t_now - (double)sample_at(slot, b, p, k)[AFO_T];
                    age += a > 0.0 ? a : 0.0;
                }
            }
        sgs += 0.5 * (r[AFO_TGX] + r[AFO_TGY]) * ne;
        sgt += r[AFO_TGT] * ne;
        nonempty += ne;
        if (r[AFO_TN] > 0.0) {
            sage += age / r[AFO_TN];
            nage += 1.0;
        }
    }
    for (int t = 0; t < nt; ++t) {
        int tx = t % ntx, ty = t / ntx;
        int x0 = tx * S, y0 = ty * S;
        int x1 = x0 + S < W ? x0 + S : W, y1 = y0 + S < H ? y0 + S : H;
        double A = (double)(x1 - x0) * (y1 - y0);
        const double *r = tiles + (size_t)t * AFO_NT;
        double e = 0.0;
        if (sv > 0.0) e += kappa * r[AFO_TVARL] / sv;
        if (su > 0.0) e += lambda * r[AFO_TU] / su;
        if (occluded && so > 0.0) e += (1.0 - kappa - lambda) * (occluded[t] / (A * b)) / so;
        E[t] = A * e;
    }
    double dcds = nonempty > 0.0 ? sgs / nonempty : 0.0;
    double dcdt = nonempty > 0.0 ? sgt / nonempty : 0.0;
    double T = nage > 0.0 ? sage / nage : 0.0;
    double Sw = importance * dcdt * T / (dcds > eps ? dcds : eps);
    double P = (double)W * H;
    double N = Sw > 0.0 ? P / (Sw * Sw) : P;
    if (N < 1.0) N = 1.0;
    if (N > P) N = P;
    gain[0] = dcds;
    gain[1] = dcdt;
    gain[2] = T;
    gain[3] = Sw;
    gain[4] = N;
}

/* ------------------------------------------------------------------------ */
/* Section 6.2: splat sizes follow the previous image's coverage map. A region
 * keeps the mean size used there, grows it fourfold where a pixel received
 * fewer than 4 samples and shrinks it by 0.7 where more than 32 reached it. */
void afo_coverage_update(int W, int H, const float *r_prev, const int32_t *n_prev,
                         float r_min, float r_max, float *r_next, int32_t *R_next)
{
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            float sum = 0.0f;
            int cnt = 0;
            for (int dj = -1; dj <= 1; ++dj)
                for (int di = -1; di <= 1; ++di) {
                    int qi = i + di, qj = j + dj;
                    if (qi < 0 || qj < 0 || qi >= W || qj >= H) continue;
                    sum = sum + r_prev[(size_t)qj * W + qi];
                    ++cnt;
                }
            size_t p = (size_t)j * W + i;
            float mean = sum / (float)cnt;
            int32_t n = n_prev[p];
            float f = n < 0 ? 1.0f : n < 4 ? 4.0f : n > 32 ? 0.7f : 1.0f;
            float r = mean * f;
            if (r < r_min) r = r_min;
            if (r > r_max) r = r_max;
            r_next[p] = r;
            R_next[p] = (int32_t)floorf(r + 0.5f);
        }
}

void afo_coverage_count(int W, int H, const int32_t *Rp, const uint32_t *off, int32_t *n)
{
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            int R = Rp[(size_t)j * W + i];
            int64_t c = 0;
            for (int dj = -R; dj <= R; ++dj)
                for (int di = -R; di <= R; ++di) {
                    int qi = i + di, qj = j + dj;
                    if (di * di + dj * dj > R * R || qi < 0 || qj < 0 || qi >= W || qj >= H) continue;
                    size_t q = (size_t)qj * W + qi;
                    c += off[q + 1] - off[q];
                }
            n[(size_t)j * W + i] = (int32_t)c;
        }
}

void afo_filter_var(int W, int H, const int32_t *Rp, const uint32_t *off, const float *rec,
                    float t_now, const double *sig_s, const double *sig_t,
                    const int64_t *pixels, int64_t n_pixels, double *out)
{
    if (pixels) {
        for (int64_t k = 0; k < n_pixels; ++k) {
            int64_t p = pixels[k];
            filter_pixel(W, H, Rp[p], off, rec, t_now, sig_s[p], sig_t[p], (int)(p % W),
                         (int)(p / W), out + p * 4);
        }
        return;
    }
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            size_t p = (size_t)j * W + i;
            filter_pixel(W, H, Rp[p], off, rec, t_now, sig_s[p], sig_t[p], i, j, out + p * 4);
        }
}

void afo_filter_brute_var(int W, int H, const int32_t *Rp, int64_t n, const float *rec,
                          float t_now, const double *sig_s, const double *sig_t, double *out)
{
    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            size_t p = (size_t)j * W + i;
            int R = Rp[p];
            double cx = i + 0.5, cy = j + 0.5, acc[4] = {0.0, 0.0, 0.0, 0.0};
            for (int64_t e = 0; e < n; ++e) {
                const float *r = rec + (size_t)e * AFO_NR;
                int qi = (int)floorf(r[AFO_RX]), qj = (int)floorf(r[AFO_RY]);
                if ((qi - i) * (qi - i) + (qj - j) * (qj - j) > R * R) continue;
                double dx = (double)r[AFO_RX] - cx, dy = (double)r[AFO_RY] - cy;
                double a = (double)t_now - (double)r[AFO_RT];
                double w = gauss_weight(dx * dx + dy * dy, a, sig_s[p], sig_t[p]);
                acc[0] += w * r[AFO_RR];
                acc[1] += w * r[AFO_RG];
                acc[2] += w * r[AFO_RB];
                acc[3] += w;
            }
            for (int c = 0; c < 3; ++c) out[p * 4 + c] = acc[3] > 0.0 ? acc[c] / acc[3] : 0.0;
            out[p * 4 + 3] = acc[3];
        }
}

/* ------------------------------------------------------------------------ */
/* Adjoint. C_p = sum_s w_ps c_s / W_p, so dC_p/dc_s = w_ps / W_p. A width
 * sigma moves every weight of the pixel: dw/dsigma_s = w d^2 / sigma_s^3 and
 * dw/dsigma_t = w a^2 / sigma_t^3, so dC_p/dsigma = (sum dw c - C_p sum dw) / W_p.
 * Each width reaches theta through its clamp: a width at its upper clamp
 * passes its gradient to the clamp; one strictly between the bounds passes it
 * to the scale (times the extent) and the offset; one at the lower bound
 * passes nothing. The gradients and the density are held fixed. */
void afo_backward(int W, int H, int b, int S, int R, const int32_t *count,
                  const double *Gx, const double *Gy, const double *Gt,
                  const double *theta, double window, double eps,
                  const uint32_t *off, const float *rec, float t_now,
                  const double *grad_rgb, double *grad_col, double *grad_theta)
{
    (void)b;
    int ntiles = ((W + S - 1) / S) * ((H + S - 1) / S);
    double *nt = (double *)malloc(sizeof(double) * ntiles);
    double *at = (double *)malloc(sizeof(double) * ntiles);
    tile_counts(W, H, S, count, nt, at);
    for (int k = 0; k < AFO_NP; ++k) grad_theta[k] = 0.0;
    for (uint32_t e = 0; e < off[(size_t)W * H]; ++e)
        grad_col[3 * (size_t)e] = grad_col[3 * (size_t)e + 1] = grad_col[3 * (size_t)e + 2] = 0.0;

    for (int j = 0; j < H; ++j)
        for (int i = 0; i < W; ++i) {
            size_t p = (size_t)j * W + i;
            Widths wd = widths_at(volume_at(i, j, W, S, nt, at, window), Gx[p], Gy[p], Gt[p],
                                  theta, eps);
            double ss = wd.sig_s, st = wd.sig_t, cx = i + 0.5, cy = j + 0.5;
            double sw = 0.0, sc[3] = {0, 0, 0}, ds = 0.0, dsc[3] = {0, 0, 0}, dt = 0.0,
                   dtc[3] = {0, 0, 0};
            for (int pass = 0; pass < 2; ++pass)
                for (int dj = -R; dj <= R; ++dj)
                    for (int di = -R; di <= R; ++di) {
                        int qi = i + di, qj = j + dj;
                        if (di * di + dj * dj > R * R || qi < 0 || qj < 0 || qi >= W || qj >= H)
                            continue;
                        size_t q = (size_t)qj * W + qi;
                        for (uint32_t e = off[q]; e < off[q + 1]; ++e) {
                            const float *r = rec + (size_t)e * AFO_NR;
                            double dx = (double)r[AFO_RX] - cx, dy = (double)r[AFO_RY] - cy;
                            double d2 = dx * dx + dy * dy;
                            double a = (double)t_now - (double)r[AFO_RT];
                            double w = gauss_weight(d2, a, ss, st);
                            double c[3] = {r[AFO_RR], r[AFO_RG], r[AFO_RB]};
                            if (pass == 0) {
                                double ws = w * d2 / (ss * ss * ss), wt = w * a * a / (st * st * st);
                                sw += w;
                                ds += ws;
                                dt += wt;
                                for (int ch = 0; ch < 3; ++ch) {
                                    sc[ch] += w * c[ch];
                                    dsc[ch] += ws * c[ch];
                                    dtc[ch] += wt * c[ch];
                                }
                            } else if (sw > 0.0) {
                                for (int ch = 0; ch < 3; ++ch)
                                    grad_col[3 * (size_t)e + ch] += grad_rgb[3 * p + ch] * w / sw;
                            }
                        }
                    }
            if (!(sw > 0.0)) continue;
            double gs = 0.0, gt = 0.0;
            for (int ch = 0; ch < 3; ++ch) {
                double C = sc[ch] / sw;
                gs += grad_rgb[3 * p + ch] * (dsc[ch] - C * ds) / sw;
                gt += grad_rgb[3 * p + ch] * (dtc[ch] - C * dt) / sw;
            }
            double lo_s = wd.raw_s > 0.5 ? wd.raw_s : 0.5;
            if (lo_s >= theta[AFO_CLAMP_S]) {
                grad_theta[AFO_CLAMP_S] += gs;
            } else if (wd.raw_s > 0.5) {
                grad_theta[AFO_ALPHA_S] += gs * wd.es;
                grad_theta[AFO_BETA_S] += gs;
            }
            double lo_t = wd.raw_t > 0.05 ? wd.raw_t : 0.05;
            if (lo_t >= theta[AFO_CLAMP_T]) {
                grad_theta[AFO_CLAMP_T] += gt;
            } else if (wd.raw_t > 0.05) {
                grad_theta[AFO_ALPHA_T] += gt * wd.et;
                grad_theta[AFO_BETA_T] += gt;
            }
        }
    free(nt);
    free(at);
}

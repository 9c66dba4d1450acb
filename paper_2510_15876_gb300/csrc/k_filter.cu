// k_filter.cu -- sections 5.1 and 5.2: filter widths from density and
// gradients, the normalised space-time Gaussian gather over each pixel's
// integer disc of frame bins, and its adjoint.
//
// Exponent shift. Every weight is 2^-E with E = d^2 ks + a^2 kt >= 0
// (ks = log2 e / (2 sigma_s^2), kt = log2 e / (2 sigma_t^2)). A pixel whose
// samples are all old under a narrow temporal filter has every E far above
// the FP32 range, so the kernel subtracts a per-pixel shift m: the minimum
// over the footprint's bins of a lower bound of E in that bin (the bin's
// nearest point to the pixel centre and its smallest a^2). Then E - m >= 0
// for every sample and E - m <= ((R+1)^2 - R^2 + ...) ks stays small for
// the sample that attains the bound, so the normalised colour is exact up to
// rounding whatever the ages; W is reported as S * 2^-m.
#include "afr_internal.cuh"

namespace afr {
namespace {

struct Widths {
    float es, et, raw_s, raw_t, ss, st;
};

__device__ __forceinline__ Widths widths(float4 g, float V, float eps, const AfrParams &prm) {
    Widths w;
    float Gs = fmaxf(0.5f * (g.x + g.y), eps);
    float Gt = fmaxf(g.z, eps);
    w.es = cbrtf(V * Gt / Gs);
    w.et = cbrtf(V * (Gs * Gs) / (Gt * Gt));
    w.raw_s = fmaf(prm.alpha_s, w.es, prm.beta_s);
    w.raw_t = fmaf(prm.alpha_t, w.et, prm.beta_t);
    w.ss = fminf(fmaxf(w.raw_s, kSigmaSMin), prm.clamp_s);
    w.st = fminf(fmaxf(w.raw_t, kSigmaTMin), prm.clamp_t);
    return w;
}

__device__ __forceinline__ float tile_volume(int x, int y, int W, int H, int S, int ntx, float window,
                                             const TilePartial *__restrict__ tiles) {
    int tx = x / S, ty = y / S;
    float A = (float)(min(S, W - tx * S) * min(S, H - ty * S));
    float n = (float)__ldg(&tiles[ty * ntx + tx].n);   // an integer count
    return n > 0.f ? A * window / n : A * window;
}

__device__ __forceinline__ int half_width(int R, int dy) {
    int h = 0;
    while ((h + 1) * (h + 1) + dy * dy <= R * R) ++h;
    return h;
}

__device__ __forceinline__ float bin_gap(int d) {   // nearest distance from a pixel centre to a bin d away
    float g = fabsf((float)d) - 0.5f;
    return g > 0.f ? g : 0.f;
}

struct PixelFrame {
    float cx, cy, ks, kt, m;
    bool any;
};

// Per-pixel constants of the gather: centre, exponent scales and shift.
__device__ __forceinline__ PixelFrame pixel_frame(int x, int y, int W, int H, int R, float2 sg,
                                                  const uint32_t *__restrict__ amin2) {
    PixelFrame f;
    f.cx = (float)x + 0.5f;
    f.cy = (float)y + 0.5f;
    f.ks = kLog2e / (2.f * sg.x * sg.x);
    f.kt = kLog2e / (2.f * sg.y * sg.y);
    float m = INFINITY;
    for (int dy = -R; dy <= R; ++dy) {
        int row = y + dy;
        if (row < 0 || row >= H) continue;
        int hw = half_width(R, dy);
        int x0 = max(0, x - hw), x1 = min(W - 1, x + hw);
        float gy = bin_gap(dy);
        for (int bx = x0; bx <= x1; ++bx) {
            uint32_t a2 = __ldg(amin2 + (size_t)row * W + bx);
            if (a2 == 0x7f800000u) continue;   // empty bin
            float gx = bin_gap(bx - x);
            float lb = fmaf(fmaf(gx, gx, gy * gy), f.ks, __uint_as_float(a2) * f.kt);
            m = fminf(m, lb);
        }
    }
    f.any = m < INFINITY;
    f.m = f.any ? m : 0.f;
    return f;
}

__device__ __forceinline__ float shifted_exponent(const PixelFrame &f, float4 r) {
    float dx = r.x - f.cx, dy = r.y - f.cy;
    float d2 = fmaf(dx, dx, dy * dy);
    return fmaf(d2, f.ks, fmaf(r.z, f.kt, -f.m));
}

// Filter widths of every pixel (unless KEEP: the widths already in the map
// are used) and the pixel's gather constants for the filter: -ks, -kt, the
// exponent shift m and the footprint radius (the configured R, or with ADAPT
// floor(r + 1/2) of the pixel's adaptive radius r, whose sample count is then
// recorded for the next update).
template <bool KEEP, bool ADAPT>
__global__ void __launch_bounds__(256) k_sigma(int W, int H, int R, int S, int ntx, float window, float eps,
                                               AfrParams prm, const float4 *__restrict__ grad,
                                               const TilePartial *__restrict__ tiles,
                                               const uint32_t *__restrict__ amin2, const float *__restrict__ radius,
                                               const uint32_t *__restrict__ foff, int32_t *__restrict__ cov_n,
                                               float2 *__restrict__ sigma, float4 *__restrict__ fconst) {
    int P = W * H;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        int x = p % W, y = p / W;
        float2 sg;
        if (KEEP) {
            sg = sigma[p];
        } else {
            Widths w = widths(__ldg(grad + p), tile_volume(x, y, W, H, S, ntx, window, tiles), eps, prm);
            sg = make_float2(w.ss, w.st);
            sigma[p] = sg;
        }
        int Rp = R;
        if (ADAPT) {
            Rp = (int)floorf(__fadd_rn(__ldg(radius + p), 0.5f));
            int32_t n = 0;
            for (int dy = -Rp; dy <= Rp; ++dy) {
                const int row = y + dy;
                if (row < 0 || row >= H) continue;
                const int hw = half_width(Rp, dy);
                const int x0 = max(0, x - hw), x1 = min(W - 1, x + hw);
                n += (int32_t)(__ldg(foff + (size_t)row * W + x1 + 1) - __ldg(foff + (size_t)row * W + x0));
            }
            cov_n[p] = n;
        }
        PixelFrame f = pixel_frame(x, y, W, H, Rp, sg, amin2);
        fconst[p] = make_float4(-f.ks, -f.kt, f.m, __int_as_float(Rp));
    }
}

// Section 6.2 in gather form: the next footprint radius of each pixel is the
// mean of the previous radii over its 3x3 neighbourhood (clipped at the
// border), times 4 below 4 samples, times 0.7 above 32 (no count: times 1),
// clamped; single precision with one rounding per operation, in the same
// order as a plain loop over the neighbourhood rows.
__global__ void __launch_bounds__(256) k_coverage_update(int W, int H, const float *__restrict__ r_prev,
                                                         const int32_t *__restrict__ n_prev, float r_min,
                                                         float r_max, float *__restrict__ r_next) {
    int P = W * H;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        const int x = p % W, y = p / W;
        float sum = 0.f;
        int cnt = 0;
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                const int qx = x + dx, qy = y + dy;
                if (qx < 0 || qy < 0 || qx >= W || qy >= H) continue;
                sum = __fadd_rn(sum, __ldg(r_prev + (size_t)qy * W + qx));
                ++cnt;
            }
        const float mean = __fdiv_rn(sum, (float)cnt);
        const int32_t n = n_prev[p];
        const float f = n < 0 ? 1.f : n < 4 ? 4.f : n > 32 ? 0.7f : 1.f;
        float r = __fmul_rn(mean, f);
        if (r < r_min) r = r_min;
        if (r > r_max) r = r_max;
        r_next[p] = r;
    }
}

__global__ void k_coverage_init(int P, float r0, float *__restrict__ r, int32_t *__restrict__ n) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
        r[p] = r0;
        n[p] = -1;
    }
}

// Forward gather. One warp owns a 2x2 block of pixels. The union of the four
// discs is, row by row of bins, one contiguous run of columns, and the frame
// view stores the records of consecutive bins of a row contiguously; so the
// union's records are (2R + 2) contiguous index ranges. Lanes enumerate the
// rows (range and count), a warp scan lays them out in one flat index space,
// and the gather runs a flat loop over it: lane l takes flat indices l,
// l + 32, ... (two independent streams per iteration), following its row with
// a cursor, so loads are coalesced and every lane runs the same trip count
// whatever the bin occupancy. A table in shared memory gives, for each
// (row, column) of the union box, the exponent shift of each of the four
// pixels, or -inf (weight 0) where the bin lies outside that pixel's disc;
// a record's column is stored with it. The arithmetic runs on pixel pairs
// (same row) with paired FP32 instructions. Each lane accumulates the four
// pixels; the warp reduces them at the end. The per-pixel constants (-ks,
// -kt, shift) come from k_sigma.
constexpr int kMaxRows = 2 * 8 + 2;   // union rows (and columns) for R <= 8
constexpr int kWarps = 8;
constexpr int kMaxBatch = 64;         // contexts per batched launch

typedef unsigned long long f2;   // two floats in one 64-bit register pair

__device__ __forceinline__ f2 pk(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ uint32_t warp_incl_scan_u(uint32_t v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Reduces 16 per-lane values across the warp; afterwards lane l holds the
// total of value ((l>>4)&1)*8 + ((l>>3)&1)*4 + ((l>>2)&1)*2 + ((l>>1)&1)
// (transposed butterfly: 8 + 4 + 2 + 1 + 1 exchanges).
__device__ __forceinline__ float warp_reduce16(float (&v)[16]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        bool hi = lane & 16;
        float send = hi ? v[k] : v[k + 8];
        float keep = hi ? v[k + 8] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        bool hi = lane & 8;
        float send = hi ? v[k] : v[k + 4];
        float keep = hi ? v[k + 4] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        bool hi = lane & 4;
        float send = hi ? v[k] : v[k + 2];
        float keep = hi ? v[k + 2] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    {
        bool hi = lane & 2;
        float send = hi ? v[0] : v[1];
        float keep = hi ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
    return v[0];
}

// Pixel pair j (pixels (0, j) and (1, j)) constants and accumulators.
struct PairConsts {
    f2 cx;         // (cx0, cx1)
    f2 cy;         // (cy0, cy1): row centres
    f2 nks[2], nkt[2];
};
struct PairAcc {
    f2 S[2], C[2], r[2], g[2], b[2];
};

// sh: the exponent shifts of the four pixels for the record's bin (-inf
// outside a pixel's disc), pixel k = 2 j + column in component k.
template <bool KAHAN>
__device__ __forceinline__ void accumulate(const PairConsts &pc, float4 sh, float4 rec, float3 c, PairAcc &A) {
    const f2 dx = sub2(pk(rec.x, rec.x), pc.cx);
    const f2 sx = mul2(dx, dx);
    const f2 dy = sub2(pk(rec.y, rec.y), pc.cy);
    const f2 sy = mul2(dy, dy);
    float sy0, sy1;
    upk(sy, sy0, sy1);
    const f2 a2 = pk(rec.z, rec.z);
    const f2 cr = pk(c.x, c.x), cg = pk(c.y, c.y), cb = pk(c.z, c.z);
    const f2 m[2] = {pk(sh.x, sh.y), pk(sh.z, sh.w)};
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const float syj = j ? sy1 : sy0;
        const f2 d2 = add2(sx, pk(syj, syj));
        const f2 e = fma2(d2, pc.nks[j], fma2(a2, pc.nkt[j], m[j]));
        float e0, e1;
        upk(e, e0, e1);
        const f2 w = pk(ex2(e0), ex2(e1));
        if (KAHAN) {
            const f2 y = sub2(w, A.C[j]);
            const f2 t = add2(A.S[j], y);
            A.C[j] = sub2(sub2(t, A.S[j]), y);
            A.S[j] = t;
        } else {
            A.S[j] = add2(A.S[j], w);
        }
        A.r[j] = fma2(w, cr, A.r[j]);
        A.g[j] = fma2(w, cg, A.g[j]);
        A.b[j] = fma2(w, cb, A.b[j]);
    }
}

// Per-warp shared memory of one 2x2 block.
struct QuadSmem {
    float4 shift[kMaxRows * kMaxRows];   // per (row, column) of the union box
    uint32_t rstart[kMaxRows + 1];       // flat index of each row's first record; rstart[nv] = total
    uint32_t rbase[kMaxRows];            // record index minus flat index within the row
};

// Row cursor of one gather stream: flat index j lies in union row v.
struct Cursor {
    int v, tb;            // row, shift-table offset of column 0 of the image
    uint32_t end, base;   // flat end of row v, record index - flat index
};

__device__ __forceinline__ void advance(Cursor &k, uint32_t j, const QuadSmem &sm, int span, int colofs) {
    while (j >= k.end) {
        ++k.v;
        k.end = sm.rstart[k.v + 1];
        k.base = sm.rbase[k.v];
        k.tb = k.v * span + colofs;
    }
}

// One 2x2 pixel block (top-left pixel bx, by) by one warp.
// VAR: each pixel's footprint radius is read from its gather constants
// (adaptive footprints); otherwise every pixel uses Rfix.
template <int CT, bool KAHAN, bool VAR>
__device__ __forceinline__ void filter_block(int W, int H, int Rfix, int bx, int by, const float4 *__restrict__ fconst,
                                             const uint32_t *__restrict__ foff, const float4 *__restrict__ fpos,
                                             const void *__restrict__ fcol, float4 *__restrict__ out,
                                             QuadSmem &sm, const DebugCheck &dc) {
    using CS = ColorStore<CT>;
    const int lane = threadIdx.x & 31;
    float4 fc = make_float4(0.f, 0.f, 0.f, __int_as_float(-1));   // -1: no pixel
    if (lane < 4) {
        const int x = bx + (lane & 1), y = by + (lane >> 1);
        if (x < W && y < H) fc = __ldg(fconst + (size_t)y * W + x);
    }
    float nks[4], nkt[4], mk[4];
    int Rk[4];   // footprint radius of each pixel, -1 outside the image
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        nks[k] = __shfl_sync(0xffffffffu, fc.x, k);
        nkt[k] = __shfl_sync(0xffffffffu, fc.y, k);
        mk[k] = __shfl_sync(0xffffffffu, fc.z, k);
        if (VAR) Rk[k] = __shfl_sync(0xffffffffu, __float_as_int(fc.w), k);
        else Rk[k] = (bx + (k & 1) < W && by + (k >> 1) < H) ? Rfix : -1;
    }
    const int R = VAR ? max(max(Rk[0], Rk[1]), max(Rk[2], Rk[3])) : Rfix;   // the block's largest footprint
    const int span = 2 * R + 2, nv = span;
    // union rows: lane v (< nv) takes bin row by + v - R; the union of the
    // four discs' rows is one run of columns [bx + lo, bx + hi]
    uint32_t cnt = 0, first = 0;
    if (lane < nv) {
        const int v = lane - R, row = by + v;
        int lo = 1 << 20, hi = -(1 << 20);
        if (VAR) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int dv = v - (k >> 1);
                if (Rk[k] >= 0 && dv >= -Rk[k] && dv <= Rk[k]) {
                    const int h = half_width(Rk[k], dv);
                    lo = min(lo, (k & 1) - h);
                    hi = max(hi, (k & 1) + h);
                }
            }
        } else {
            // two pixel rows, one radius: the union row spans the wider half-width
            const bool col1 = bx + 1 < W, row1 = by + 1 < H;
            const int h0 = (v >= -R && v <= R) ? half_width(R, v) : -1;
            const int h1 = (row1 && v - 1 >= -R && v - 1 <= R) ? half_width(R, v - 1) : -1;
            const int hm = max(h0, h1);
            if (hm >= 0) {
                lo = -hm;
                hi = (col1 ? 1 : 0) + hm;
            }
        }
        if (lo <= hi && row >= 0 && row < H) {
            const int c0 = max(0, bx + lo), c1 = min(W - 1, bx + hi);
            const size_t q = (size_t)row * W;
            first = __ldg(foff + q + c0);
            cnt = __ldg(foff + q + c1 + 1) - first;
            if (!AFR_CHECK(__ldg(foff + q + c1 + 1) >= first && cnt <= dc.cap, dc.derr)) cnt = 0;
        }
    }
    const uint32_t incl = warp_incl_scan_u(cnt);
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    if (lane < nv) {
        sm.rstart[lane + 1] = incl;
        sm.rbase[lane] = first - (incl - cnt);
    }
    if (lane == 0) sm.rstart[0] = 0;
    // shift table: entry (v, u) of pixel k = (kx, ky) is its shift if
    // (u - kx)^2 + (v - ky)^2 <= R_k^2 (the pixel's own disc; none outside
    // the image)
    for (int t = lane; t < nv * span; t += 32) {
        const int v = t / span - R, u = t % span - R;
        float s4[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int du = u - (k & 1), dv = v - (k >> 1);
            s4[k] = (Rk[k] >= 0 && du * du + dv * dv <= Rk[k] * Rk[k]) ? mk[k] : -INFINITY;
        }
        sm.shift[t] = make_float4(s4[0], s4[1], s4[2], s4[3]);
    }
    __syncwarp();
    PairConsts pc;
    pc.cx = pk((float)bx + 0.5f, (float)bx + 1.5f);
    pc.cy = pk((float)by + 0.5f, (float)by + 1.5f);
    pc.nks[0] = pk(nks[0], nks[1]);
    pc.nks[1] = pk(nks[2], nks[3]);
    pc.nkt[0] = pk(nkt[0], nkt[1]);
    pc.nkt[1] = pk(nkt[2], nkt[3]);
    PairAcc A;
#pragma unroll
    for (int j = 0; j < 2; ++j) A.S[j] = A.C[j] = A.r[j] = A.g[j] = A.b[j] = 0ull;
    const int colofs = R - bx;   // table column of image column qx: qx + colofs
    Cursor ka{-1, 0, 0u, 0u}, kb{-1, 0, 0u, 0u};
    uint32_t j = lane;
    for (; j + 32 < total; j += 64) {
        advance(ka, j, sm, span, colofs);
        advance(kb, j + 32, sm, span, colofs);
        uint32_t ia = j + ka.base, ib = j + 32 + kb.base;
        const bool va = AFR_CHECK(ia < dc.cap, dc.derr), vb = AFR_CHECK(ib < dc.cap, dc.derr);
        if (!va) ia = 0;   // skipped: record 0 read, weight 0
        if (!vb) ib = 0;
        const float4 ra = __ldg(fpos + ia), rb = __ldg(fpos + ib);
        const float3 ca = CS::load(fcol, ia), cbv = CS::load(fcol, ib);
        int ta = ka.tb + __float_as_int(ra.w), tb = kb.tb + __float_as_int(rb.w);
        const bool wa = va && AFR_CHECK(ta >= 0 && ta < kMaxRows * kMaxRows, dc.derr);
        const bool wb = vb && AFR_CHECK(tb >= 0 && tb < kMaxRows * kMaxRows, dc.derr);
        if (!wa) ta = 0;
        if (!wb) tb = 0;
        float4 sa = sm.shift[ta], sb = sm.shift[tb];
        if (!wa) sa = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
        if (!wb) sb = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
        accumulate<KAHAN>(pc, sa, ra, ca, A);
        accumulate<KAHAN>(pc, sb, rb, cbv, A);
    }
    if (j < total) {
        advance(ka, j, sm, span, colofs);
        uint32_t ia = j + ka.base;
        const bool va = AFR_CHECK(ia < dc.cap, dc.derr);
        if (!va) ia = 0;
        const float4 ra = __ldg(fpos + ia);
        int ta = ka.tb + __float_as_int(ra.w);
        const bool wa = va && AFR_CHECK(ta >= 0 && ta < kMaxRows * kMaxRows, dc.derr);
        if (!wa) ta = 0;
        float4 sa = sm.shift[ta];
        if (!wa) sa = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY);
        accumulate<KAHAN>(pc, sa, ra, CS::load(fcol, ia), A);
    }
    float vals[16];
#pragma unroll
    for (int jj = 0; jj < 2; ++jj) {
        float a, b;
        upk(KAHAN ? sub2(A.S[jj], A.C[jj]) : A.S[jj], a, b);
        vals[2 * jj] = a;
        vals[2 * jj + 1] = b;
        upk(A.r[jj], a, b);
        vals[4 + 2 * jj] = a;
        vals[4 + 2 * jj + 1] = b;
        upk(A.g[jj], a, b);
        vals[8 + 2 * jj] = a;
        vals[8 + 2 * jj + 1] = b;
        upk(A.b[jj], a, b);
        vals[12 + 2 * jj] = a;
        vals[12 + 2 * jj + 1] = b;
    }
    const float tot = warp_reduce16(vals);
    // value qq*4 + k (qq: S, r, g, b) of pixel k moves to lane k
    float q[4];
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
        const int want = qq * 4 + (lane & 3);
        const int src = ((want >> 3) & 1) * 16 + ((want >> 2) & 1) * 8 + ((want >> 1) & 1) * 4 + (want & 1) * 2;
        q[qq] = __shfl_sync(0xffffffffu, tot, src);
    }
    if (lane < 4 && bx + (lane & 1) < W && by + (lane >> 1) < H) {
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
        if (q[0] > 0.f) {
            const float inv = 1.f / q[0];
            o = make_float4(q[1] * inv, q[2] * inv, q[3] * inv, q[0] * ex2(-fc.z));
        }
        out[(size_t)(by + (lane >> 1)) * W + bx + (lane & 1)] = o;
    }
    __syncwarp();
}

// Tile of (2 * tbx) x (2 * 32 / tbx) pixels per CTA: 32 blocks of 2x2, four
// per warp.
template <int CT, bool KAHAN, bool VAR>
__global__ void __launch_bounds__(256, 3) k_filter(int W, int H, int R, int tbx, const float4 *__restrict__ fconst,
                                                   const uint32_t *__restrict__ foff, const float4 *__restrict__ fpos,
                                                   const void *__restrict__ fcol, float4 *__restrict__ out,
                                                   DebugCheck dc) {
    __shared__ QuadSmem smem[kWarps];
    const int warp = threadIdx.x >> 5;
    const int tby = 32 / tbx;
    for (int blk = warp; blk < 32; blk += kWarps) {
        const int bx = blockIdx.x * 2 * tbx + (blk % tbx) * 2, by = blockIdx.y * 2 * tby + (blk / tbx) * 2;
        if (bx >= W || by >= H) continue;   // warp-uniform
        filter_block<CT, KAHAN, VAR>(W, H, R, bx, by, fconst, foff, fpos, fcol, out, smem[warp], dc);
    }
}

// ---- batched form ---------------------------------------------------------------
// Two launches reconstruct many contexts. k_batch_sigma computes the widths
// and gather constants of every pixel of every context (thread per pixel,
// full occupancy: the per-pixel work is bound by the latency of the footprint
// loads). k_batch, a persistent kernel, then takes tiles of (2 tbx) x
// (64 / tbx) pixels of any context from a work queue (one atomic counter, the
// next tile claimed while the current one runs), largest contexts first, and
// filters them. Tiles never wait for one another.

// owning context of a batch-wide index: the last c with first[c] <= v
__device__ __forceinline__ int batch_owner(const uint32_t *first, int nctx, uint32_t v) {
    int lo = 0, hi = nctx - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (first[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Widths of every pixel of the batch: each block takes chunks of
// kBatchSigmaChunk pixels of one context (chunks are numbered per context from
// BatchCtx::s0) and reads the context's record once per chunk.
__global__ void __launch_bounds__(256) k_batch_sigma(const BatchCtx *__restrict__ cs, int nctx, uint32_t nchunks) {
    __shared__ uint32_t first[kMaxBatch];      // first chunk of each context
    __shared__ BatchCtx ctx;
    for (int c = threadIdx.x; c < nctx; c += blockDim.x) first[c] = cs[c].s0;
    __syncthreads();
    for (uint32_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
        if (threadIdx.x == 0) ctx = cs[batch_owner(first, nctx, ch)];
        __syncthreads();
        const int W = ctx.W, H = ctx.H, P = W * H;
        const int p0 = (int)(ch - ctx.s0) * kBatchSigmaChunk, p1 = min(P, p0 + kBatchSigmaChunk);
        for (int p = p0 + (int)threadIdx.x; p < p1; p += blockDim.x) {
            const int px = p % W, py = p / W;
            Widths w = widths(__ldg(ctx.grad + p), tile_volume(px, py, W, H, ctx.S, ctx.ntx, ctx.window, ctx.tiles),
                              ctx.eps, ctx.prm);
            const float2 sg = make_float2(w.ss, w.st);
            ctx.sigma[p] = sg;
            const PixelFrame f = pixel_frame(px, py, W, H, ctx.R, sg, ctx.amin2);
            ctx.fconst[p] = make_float4(-f.ks, -f.kt, f.m, __int_as_float(ctx.R));
        }
        __syncthreads();
    }
}

template <int CT, bool KAHAN>
__global__ void __launch_bounds__(256, 3) k_batch(const BatchCtx *__restrict__ cs, int nctx, uint32_t total,
                                                  uint32_t *queue) {
    // shared memory: the per-warp tables and two words, so that three CTAs
    // fit the 132 KB shared-memory carve-out and leave the rest to L1
    __shared__ QuadSmem smem[kWarps];
    __shared__ uint32_t item_buf[2];            // current and next claimed tile
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) item_buf[0] = atomicAdd(queue, 1u);
    __syncthreads();
    for (int it = 0;; ++it) {
        const uint32_t item = item_buf[it & 1];
        if (item >= total) break;
        if (threadIdx.x == 0) item_buf[(it + 1) & 1] = atomicAdd(queue, 1u);
        int lo = 0, hi = nctx - 1;                  // owning context: last c with cs[c].a0 <= item
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(&cs[mid].a0) <= item) lo = mid;
            else hi = mid - 1;
        }
        const BatchCtx &x = cs[lo];
        const uint32_t local = item - x.a0;
        const int band = (int)(local / (uint32_t)x.ntiles_x), tile = (int)(local % (uint32_t)x.ntiles_x);
        const int tbx = x.tbx, tw = 2 * tbx, th = 2 * (32 / tbx);
        for (int blk = warp; blk < 32; blk += kWarps) {
            const int bx = tile * tw + (blk % tbx) * 2, by = band * th + (blk / tbx) * 2;
            if (bx >= x.W || by >= x.H) continue;
            filter_block<CT, KAHAN, false>(x.W, x.H, x.R, bx, by, x.fconst, x.foff, x.fpos, x.fcol, x.out,
                                           smem[warp], DebugCheck{x.fcap, x.derr});
        }
        __syncthreads();
    }
}

// ---- adjoint -------------------------------------------------------------------

template <int CT>
__global__ void __launch_bounds__(128) k_bwd_pixel(int W, int H, int R, int S_, int ntx, float window, float eps,
                                                   AfrParams prm, const float4 *__restrict__ grad,
                                                   const TilePartial *__restrict__ tiles,
                                                   const float2 *__restrict__ sigma, const uint32_t *__restrict__ amin2,
                                                   const uint32_t *__restrict__ foff, const float4 *__restrict__ fpos,
                                                   const void *__restrict__ fcol, const float4 *__restrict__ gout,
                                                   float4 *__restrict__ bg, float4 *__restrict__ bframe,
                                                   float *__restrict__ bparam) {
    using CS = ColorStore<CT>;
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y * blockDim.y + threadIdx.y;
    float gp[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (x < W && y < H) {
        size_t p = (size_t)y * W + x;
        float2 sgm = __ldg(sigma + p);
        PixelFrame f = pixel_frame(x, y, W, H, R, sgm, amin2);
        float4 g = __ldg(gout + p);
        if (!f.any) {
            bg[p] = make_float4(0.f, 0.f, 0.f, 0.f);
            bframe[p] = make_float4(f.ks, f.kt, f.m, 0.f);
        } else {
            float S = 0.f, sc[3] = {0.f, 0.f, 0.f}, Ds = 0.f, dsc[3] = {0.f, 0.f, 0.f}, Dt = 0.f,
                  dtc[3] = {0.f, 0.f, 0.f};
            for (int dy = -R; dy <= R; ++dy) {
                int row = y + dy;
                if (row < 0 || row >= H) continue;
                int hw = half_width(R, dy);
                int x0 = max(0, x - hw), x1 = min(W - 1, x + hw);
                uint32_t e0 = __ldg(foff + (size_t)row * W + x0), e1 = __ldg(foff + (size_t)row * W + x1 + 1);
                for (uint32_t e = e0; e < e1; ++e) {
                    float4 r = __ldg(fpos + e);
                    float3 c = CS::load(fcol, e);
                    float w = ex2(-shifted_exponent(f, r));
                    float ddx = r.x - f.cx, ddy = r.y - f.cy;
                    float d2 = fmaf(ddx, ddx, ddy * ddy);
                    float ws = w * d2, wt = w * r.z;
                    S += w;
                    sc[0] = fmaf(w, c.x, sc[0]); sc[1] = fmaf(w, c.y, sc[1]); sc[2] = fmaf(w, c.z, sc[2]);
                    Ds += ws; Dt += wt;
                    dsc[0] = fmaf(ws, c.x, dsc[0]); dsc[1] = fmaf(ws, c.y, dsc[1]); dsc[2] = fmaf(ws, c.z, dsc[2]);
                    dtc[0] = fmaf(wt, c.x, dtc[0]); dtc[1] = fmaf(wt, c.y, dtc[1]); dtc[2] = fmaf(wt, c.z, dtc[2]);
                }
            }
            float inv = 1.f / S;
            float gch[3] = {g.x, g.y, g.z};
            float s3 = sgm.x * sgm.x * sgm.x, t3 = sgm.y * sgm.y * sgm.y;
            float gs = 0.f, gt = 0.f;
            for (int ch = 0; ch < 3; ++ch) {
                float C = sc[ch] * inv;
                gs = fmaf(gch[ch], (dsc[ch] - C * Ds) * inv / s3, gs);
                gt = fmaf(gch[ch], (dtc[ch] - C * Dt) * inv / t3, gt);
            }
            bg[p] = make_float4(g.x * inv, g.y * inv, g.z * inv, 1.f);
            bframe[p] = make_float4(f.ks, f.kt, f.m, 1.f);
            // chain through the width mapping; the widths depend on theta only
            Widths wd = widths(__ldg(grad + p), tile_volume(x, y, W, H, S_, ntx, window, tiles), eps, prm);
            if (fmaxf(wd.raw_s, kSigmaSMin) >= prm.clamp_s) gp[2] = gs;
            else if (wd.raw_s > kSigmaSMin) { gp[0] = gs * wd.es; gp[1] = gs; }
            if (fmaxf(wd.raw_t, kSigmaTMin) >= prm.clamp_t) gp[5] = gt;
            else if (wd.raw_t > kSigmaTMin) { gp[3] = gt * wd.et; gp[4] = gt; }
        }
    }
    // block reduction of the six parameter gradients, then one FP64 partial per block
    __shared__ float sh[6][4];
    int tid = threadIdx.y * blockDim.x + threadIdx.x;
    for (int k = 0; k < 6; ++k) {
        float v = gp[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((tid & 31) == 0) sh[k][tid >> 5] = v;
    }
    __syncthreads();
    if (tid < 6) {
        float acc = 0.f;
        for (int w = 0; w < 4; ++w) acc += sh[tid][w];
        bparam[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * 6 + tid] = acc;
    }
}

// Gradient of each frame record's colour: sum over the pixels whose disc
// holds the record's bin of (dL/dC_p / S_p) * shifted weight.
__global__ void __launch_bounds__(256) k_bwd_record(int W, int H, int R, const uint32_t *__restrict__ foff,
                                                    const float4 *__restrict__ fpos, const float4 *__restrict__ bg,
                                                    const float4 *__restrict__ bframe, float *__restrict__ gcol) {
    uint32_t n = __ldg(foff + (size_t)W * H);
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        float4 r = __ldg(fpos + e);
        int qx = (int)floorf(r.x), qy = (int)floorf(r.y);
        float a0 = 0.f, a1 = 0.f, a2 = 0.f;
        for (int dy = -R; dy <= R; ++dy) {
            int y = qy + dy;
            if (y < 0 || y >= H) continue;
            int hw = half_width(R, dy);
            for (int x = max(0, qx - hw); x <= min(W - 1, qx + hw); ++x) {
                size_t p = (size_t)y * W + x;
                float4 fr = __ldg(bframe + p);
                if (fr.w == 0.f) continue;
                PixelFrame f;
                f.cx = (float)x + 0.5f;
                f.cy = (float)y + 0.5f;
                f.ks = fr.x;
                f.kt = fr.y;
                f.m = fr.z;
                float w = ex2(-shifted_exponent(f, r));
                float4 g = __ldg(bg + p);
                a0 = fmaf(g.x, w, a0);
                a1 = fmaf(g.y, w, a1);
                a2 = fmaf(g.z, w, a2);
            }
        }
        gcol[3 * (size_t)e] = a0;
        gcol[3 * (size_t)e + 1] = a1;
        gcol[3 * (size_t)e + 2] = a2;
    }
}

// The six parameter gradients summed over the blocks' partials: one warp per
// parameter, each lane a compensated (Kahan) FP32 sum over a strided share of
// the blocks, then the 32 lane sums (value and compensation) added in a fixed
// order by lane 0.
__global__ void k_bwd_params(const float *__restrict__ part, int nblocks, float *__restrict__ out) {
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k >= 6) return;
    float s = 0.f, c = 0.f;
    for (int i = lane; i < nblocks; i += 32) {
        const float y = part[(size_t)i * 6 + k] - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __shared__ float ss[6][32], cs[6][32];
    ss[k][lane] = s;
    cs[k][lane] = c;
    __syncwarp();
    if (lane == 0) {
        float S = 0.f, C = 0.f;
        for (int l = 0; l < 32; ++l) {
            const float y = ss[k][l] - cs[k][l] - C;
            const float t = S + y;
            C = (t - S) - y;
            S = t;
        }
        out[k] = S;
    }
}

template <int CT>
__global__ void k_set_colors(const float *__restrict__ rgb, const uint32_t *__restrict__ foff, int P,
                             void *__restrict__ fcol) {
    uint32_t n = __ldg(foff + P);
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        float r = rgb[3 * (size_t)e], g = rgb[3 * (size_t)e + 1], b = rgb[3 * (size_t)e + 2];
        if (CT == AFR_F32) {
            reinterpret_cast<float4 *>(fcol)[e] = make_float4(r, g, b, 0.f);
        } else if (CT == AFR_F16) {
            reinterpret_cast<ushort4 *>(fcol)[e] = make_ushort4(__half_as_ushort(__float2half_rn(r)),
                                                                __half_as_ushort(__float2half_rn(g)),
                                                                __half_as_ushort(__float2half_rn(b)), 0);
        } else {
            reinterpret_cast<ushort4 *>(fcol)[e] = make_ushort4(__bfloat16_as_ushort(__float2bfloat16_rn(r)),
                                                                __bfloat16_as_ushort(__float2bfloat16_rn(g)),
                                                                __bfloat16_as_ushort(__float2bfloat16_rn(b)), 0);
        }
    }
}

const dim3 kFilterBlock(32, 4);
const dim3 kQuadBlock(256);

}  // namespace

cudaError_t launch_sigma(AfrContext *c, const AfrParams *prm, bool keep, bool adaptive, cudaStream_t s) {
    const int g = grid_for(c->P, 256);
    const float *radius = nullptr;
    if (adaptive) {
        float *next = c->cov_r[1 - c->cov_cur];
        k_coverage_update<<<g, 256, 0, s>>>(c->W, c->H, c->cov_r[c->cov_cur], c->cov_n, 0.5f, 8.f, next);
        c->cov_cur = 1 - c->cov_cur;
        radius = next;
    }
#define AFR_SIGMA(K, A)                                                                                         \
    k_sigma<K, A><<<g, 256, 0, s>>>(c->W, c->H, c->R, c->S, c->ntx, c->cfg.window, c->cfg.eps_grad, *prm, c->grad, \
                                    c->tiles, c->amin2, radius, c->foff, c->cov_n, c->sigma, c->fconst)
    if (keep && adaptive) AFR_SIGMA(true, true);
    else if (keep) AFR_SIGMA(true, false);
    else if (adaptive) AFR_SIGMA(false, true);
    else AFR_SIGMA(false, false);
#undef AFR_SIGMA
    return cudaGetLastError();
}

cudaError_t launch_coverage_init(AfrContext *c, cudaStream_t s) {
    k_coverage_init<<<grid_for(c->P, 256), 256, 0, s>>>(c->P, (float)c->R, c->cov_r[c->cov_cur], c->cov_n);
    return cudaGetLastError();
}

cudaError_t launch_filter(AfrContext *c, float t_now, bool adaptive, float4 *out, cudaStream_t s) {
    (void)t_now;
    const DebugCheck dc{(uint32_t)c->frame_cap, c->derr};
    const int tbx = c->tile_bx, tw = 2 * tbx, th = 2 * (32 / tbx);
    dim3 grid((c->W + tw - 1) / tw, (c->H + th - 1) / th);
#define AFR_FILTER(CT_, K_, V_)                                                                          \
    k_filter<CT_, K_, V_><<<grid, kQuadBlock, 0, s>>>(c->W, c->H, c->R, tbx, c->fconst, c->foff, c->fpos, c->fcol, \
                                                      out, dc)
    switch (c->ct) {
        case AFR_F32:
            if (adaptive) AFR_FILTER(AFR_F32, false, true);
            else AFR_FILTER(AFR_F32, false, false);
            break;
        case AFR_F16:
            if (adaptive) AFR_FILTER(AFR_F16, true, true);
            else AFR_FILTER(AFR_F16, true, false);
            break;
        default:
            if (adaptive) AFR_FILTER(AFR_BF16, true, true);
            else AFR_FILTER(AFR_BF16, true, false);
            break;
    }
#undef AFR_FILTER
    return cudaGetLastError();
}

cudaError_t launch_backward(AfrContext *c, const float4 *grad_rgb, float *grad_col, float *grad_prm,
                            cudaStream_t s) {
    dim3 grid((c->W + kFilterBlock.x - 1) / kFilterBlock.x, (c->H + kFilterBlock.y - 1) / kFilterBlock.y);
    float4 *bframe = c->bgrad + c->P;
    const AfrParams &prm = c->recon_params;
#define AFR_BWD(CT_)                                                                                        \
    k_bwd_pixel<CT_><<<grid, kFilterBlock, 0, s>>>(c->W, c->H, c->R, c->S, c->ntx, c->cfg.window,           \
                                                   c->cfg.eps_grad, prm, c->grad, c->tiles, c->sigma, c->amin2, \
                                                   c->foff, c->fpos, c->fcol, grad_rgb, c->bgrad, bframe,   \
                                                   c->bparam)
    switch (c->ct) {
        case AFR_F32: AFR_BWD(AFR_F32); break;
        case AFR_F16: AFR_BWD(AFR_F16); break;
        default: AFR_BWD(AFR_BF16); break;
    }
#undef AFR_BWD
    if (grad_col)
        k_bwd_record<<<grid_for((size_t)c->P * c->b, 256), 256, 0, s>>>(c->W, c->H, c->R, c->foff, c->fpos, c->bgrad,
                                                                        bframe, grad_col);
    if (grad_prm) k_bwd_params<<<1, 6 * 32, 0, s>>>(c->bparam, (int)(grid.x * grid.y), grad_prm);
    return cudaGetLastError();
}

cudaError_t launch_set_frame_colors(AfrContext *c, const float *rgb, cudaStream_t s) {
    int g = grid_for((size_t)c->P * c->b, 256);
    switch (c->ct) {
        case AFR_F32: k_set_colors<AFR_F32><<<g, 256, 0, s>>>(rgb, c->foff, c->P, c->fcol); break;
        case AFR_F16: k_set_colors<AFR_F16><<<g, 256, 0, s>>>(rgb, c->foff, c->P, c->fcol); break;
        default: k_set_colors<AFR_BF16><<<g, 256, 0, s>>>(rgb, c->foff, c->P, c->fcol); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_batch(int ct, const BatchCtx *cs, int nctx, uint32_t nchunks, uint32_t total, uint32_t *queue,
                         int grid, cudaStream_t s) {
    k_batch_sigma<<<grid_for((size_t)nchunks * 256, 256), 256, 0, s>>>(cs, nctx, nchunks);
    switch (ct) {
        case AFR_F32: k_batch<AFR_F32, false><<<grid, kQuadBlock, 0, s>>>(cs, nctx, total, queue); break;
        case AFR_F16: k_batch<AFR_F16, true><<<grid, kQuadBlock, 0, s>>>(cs, nctx, total, queue); break;
        default: k_batch<AFR_BF16, true><<<grid, kQuadBlock, 0, s>>>(cs, nctx, total, queue); break;
    }
    return cudaGetLastError();
}

int backward_blocks(int W, int H) {
    return (int)(((W + kFilterBlock.x - 1) / kFilterBlock.x) * ((H + kFilterBlock.y - 1) / kFilterBlock.y));
}

}  // namespace afr

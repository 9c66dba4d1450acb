"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a queue
model, closed forms, hand-worked examples, defining identities, brute force,
a scatter-order sum and finite differences. No GPU is needed.
"""
import collections
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
LUMA = (0.2126, 0.7152, 0.0722)   # Rec. 709 weights (the reading of "luminance")


def _batch(rng, n, W, H, t_sorted=True, bad_frac=0.0):
    x = rng.uniform(0, W, n).astype(np.float32)
    y = rng.uniform(0, H, n).astype(np.float32)
    t = rng.uniform(0, 1, n)
    t = np.sort(t) if t_sorted else t
    pos = np.stack([x, y, t.astype(np.float32), rng.uniform(0, 1, n).astype(np.float32)], 1)
    col = np.zeros((n, 4), np.float32)
    col[:, :3] = rng.uniform(0, 1, (n, 3))
    mo = rng.uniform(-3, 3, (n, 2)).astype(np.float32)
    if bad_frac:
        k = int(n * bad_frac)
        idx = rng.choice(n, k, replace=False)
        kinds = rng.integers(0, 6, k)
        for i, kind in zip(idx, kinds):
            if kind == 0:
                pos[i, 0] = np.nan
            elif kind == 1:
                pos[i, 0] = W          # x == W is outside [0, W)
            elif kind == 2:
                pos[i, 1] = -1e-3
            elif kind == 3:
                col[i, 1] = np.inf
            elif kind == 4:
                mo[i, 0] = np.nan
            else:
                pos[i, 2] = np.inf
    return pos, col, mo


def _single(x, y, t, rgb, mo=(0.0, 0.0), depth=0.5):
    pos = np.array([[x, y, t, depth]], np.float32)
    col = np.array([[rgb[0], rgb[1], rgb[2], 0.0]], np.float32)
    m = np.array([mo], np.float32)
    return pos, col, m


# --------------------------------------------------------------------------- ingest
@pytest.mark.parametrize("b", [1, 2, 4])
def test_ingest_matches_queue_model(b):
    """Section 4: each pixel is a queue of depth b, new samples in front, the
    back evicted when full. Compare against collections.deque(maxlen=b)."""
    rng = np.random.default_rng(b)
    W, H = 7, 5
    ring = oracle.Ring(W, H, b)
    model = [collections.deque(maxlen=b) for _ in range(W * H)]
    seq = 0
    rejected = 0
    for n in (0, 1, 37, 120, 5):
        pos, col, mo = _batch(rng, n, W, H, bad_frac=0.1 if n > 10 else 0.0)
        rej = ring.insert(pos, col, mo)
        for i in range(n):
            vals = [pos[i, 0], pos[i, 1], pos[i, 2], col[i, 0], col[i, 1], col[i, 2], mo[i, 0],
                    mo[i, 1]]
            x, y = float(pos[i, 0]), float(pos[i, 1])
            if all(math.isfinite(float(v)) for v in vals) and 0 <= x < W and 0 <= y < H:
                p = int(math.floor(y)) * W + int(math.floor(x))
                model[p].appendleft((seq + i, pos[i].copy(), col[i, :3].copy(), mo[i].copy()))
            else:
                rejected += 1
        seq += n
        assert rej >= 0
    assert ring.rejected == rejected
    for p in range(W * H):
        assert ring.count[p] == len(model[p])
        for k, (s, ps, cs, ms) in enumerate(model[p]):
            assert ring.seq[p, k] == s
            np.testing.assert_array_equal(ring.slot[p, k, 0:4], ps)
            np.testing.assert_array_equal(ring.slot[p, k, 4:7], cs)
            np.testing.assert_array_equal(ring.slot[p, k, 7:9], ms)


# --------------------------------------------------------------------------- age weight
def test_age_weight_golden():
    """Section 4: weight exp(-3.47 a), about 1/32 at age one window. A pixel
    holding L=0 at age 1 and L=1 at age 0 has mean 1/(1 + w(1))."""
    rows = [list(map(float, l.split())) for l in open(os.path.join(GOLDEN, "age_weight.txt"))
            if l.strip() and not l.startswith("#")]
    ring = oracle.Ring(1, 1, 2)
    ring.insert(*_single(0.5, 0.5, 0.0, (0, 0, 0)))
    ring.insert(*_single(0.5, 0.5, 1.0, (1, 1, 1)))
    L, *_ = oracle.gradients(ring, 1.0)
    w1 = 1.0 / L[0] - 1.0
    lo, hi = rows[0][1], rows[0][2]
    assert lo <= w1 <= hi
    assert abs(w1 - math.exp(-3.47)) < 1e-12


# --------------------------------------------------------------------------- gradients
def _grid_ring(W, H, b, color_fn, times=(0.25, 0.75)):
    ring = oracle.Ring(W, H, b)
    for t in times:
        pos, col, mo = [], [], []
        for y in range(H):
            for x in range(W):
                pos.append([x + 0.5, y + 0.5, t, 0.5])
                c = color_fn(x, y, t)
                col.append([c[0], c[1], c[2], 0.0])
                mo.append([0.0, 0.0])
        ring.insert(np.array(pos, np.float32), np.array(col, np.float32),
                    np.array(mo, np.float32))
    return ring


def test_constant_scene_has_zero_gradients():
    ring = _grid_ring(6, 5, 3, lambda x, y, t: (0.3, 0.6, 0.9), times=(0.1, 0.4, 0.8))
    L, gx, gy, gt = oracle.gradients(ring)
    np.testing.assert_allclose(
        L, sum(w * float(np.float32(c)) for w, c in zip(LUMA, (0.3, 0.6, 0.9))), rtol=1e-12)
    assert np.all(np.abs(gx) < 1e-12) and np.all(np.abs(gy) < 1e-12)
    assert np.all(np.abs(gt) < 1e-12)


@pytest.mark.parametrize("channel", [0, 1, 2, None])
def test_linear_ramp_gives_exact_spatial_gradient(channel):
    """Section 4.1: G_x is the mean one-sided |dL| over 1-pixel steps, so a
    ramp L = k x gives G_x = k everywhere (borders included) and G_y = 0. A
    single-primary ramp scales by that primary's luminance weight."""
    k = 0.0625      # exact in float32, so the ramp is exact

    def col(x, y, t):
        c = [0.0, 0.0, 0.0]
        if channel is None:
            c = [k * x] * 3
        else:
            c[channel] = k * x
        return c

    ring = _grid_ring(9, 4, 2, col)
    _, gx, gy, gt = oracle.gradients(ring)
    expect = k if channel is None else k * LUMA[channel]
    np.testing.assert_allclose(gx, expect, rtol=1e-9)
    assert np.all(np.abs(gy) < 1e-12) and np.all(np.abs(gt) < 1e-12)
    # transposed ramp
    ring = _grid_ring(4, 9, 2, lambda x, y, t: col(y, x, t))
    _, gx, gy, _ = oracle.gradients(ring)
    np.testing.assert_allclose(gy, expect, rtol=1e-9)
    assert np.all(np.abs(gx) < 1e-12)


def test_spatial_gradient_skips_empty_neighbours():
    """A side whose neighbour holds no sample is left out of the mean."""
    ring = oracle.Ring(3, 1, 2)
    ring.insert(*_single(0.5, 0.5, 0.5, (0.0, 0.0, 0.0)))
    ring.insert(*_single(1.5, 0.5, 0.5, (1.0, 1.0, 1.0)))
    _, gx, gy, _ = oracle.gradients(ring)
    np.testing.assert_allclose(gx, [1.0, 1.0, 0.0])
    np.testing.assert_allclose(gy, 0.0)


@pytest.mark.parametrize("shuffle", [False, True])
def test_linear_in_time_colour_gives_exact_temporal_gradient(shuffle):
    """Section 4.1: G_t = |dL| / dt over samples at one location; with colour
    c(t) = c0 + k t every pair gives k, so any positive weighting gives k.
    Inserting out of time order must not matter (pairs follow time)."""
    k = 0.7
    times = np.array([0.05, 0.2, 0.33, 0.61, 0.9])
    if shuffle:
        times = times[[3, 0, 4, 1, 2]]
    ring = oracle.Ring(1, 1, 8)
    for t in times:
        ring.insert(*_single(0.5, 0.5, t, (0.1 + k * t,) * 3))
    _, _, _, gt = oracle.gradients(ring)
    np.testing.assert_allclose(gt[0], k, rtol=1e-6)


def test_temporal_gradient_hand_example():
    """Three samples at one pixel, L = 1, 0, 0.5 at t = 1, 0.5, 0 (t_now = 1):
    pairs (1,0.5) and (0.5,0); weights are the newer sample's exp(-3.47 a)."""
    ring = oracle.Ring(1, 1, 4)
    for t, L in ((0.0, 0.5), (0.5, 0.0), (1.0, 1.0)):
        ring.insert(*_single(0.5, 0.5, t, (L, L, L)))
    _, _, _, gt = oracle.gradients(ring, 1.0)
    w0, w1 = 1.0, math.exp(-3.47 * 0.5)
    assert abs(gt[0] - (w0 * 1.0 + w1 * 0.5) / (w0 * 0.5 + w1 * 0.5)) < 1e-6


def test_single_sample_has_no_temporal_gradient():
    ring = oracle.Ring(2, 1, 4)
    ring.insert(*_single(0.5, 0.5, 0.3, (0.2, 0.5, 0.1)))
    L, gx, gy, gt = oracle.gradients(ring)
    assert gt[0] == 0.0 and math.isnan(L[1]) and gx[1] == 0.0


# --------------------------------------------------------------------------- tiles
def test_tile_variance_two_valued_closed_form():
    """Section 4: v = (1/n) sum (L - L_m)^2; with equal ages a tile holding a
    fraction q of L=1 and 1-q of L=0 has mean q and variance q (1 - q)."""
    W = H = 4
    ring = oracle.Ring(W, H, 4)
    rng = np.random.default_rng(0)
    ones = 0
    n = 0
    for y in range(H):
        for x in range(W):
            for _ in range(3):
                v = float(rng.integers(0, 2))
                ones += v
                n += 1
                ring.insert(*_single(x + 0.3, y + 0.7, 0.5, (v, v, v)))
    g = oracle.gradients(ring)
    st = oracle.tile_feedback(ring, g, S=4)
    q = ones / n
    assert st[0, 0] == n
    np.testing.assert_allclose(st[0, 2], q, rtol=1e-12)
    np.testing.assert_allclose(st[0, 3], q * (1 - q), rtol=1e-12)


def test_undersampling_hand_example():
    rows = [list(map(float, l.split())) for l in open(os.path.join(GOLDEN, "undersampling_hand.txt"))
            if l.strip() and not l.startswith("#")]
    ring = oracle.Ring(4, 4, 2)
    per_tile = {0: 8, 1: 0, 2: 4, 3: 6}
    for tile, n in per_tile.items():
        tx, ty = tile % 2, tile // 2
        px = [(tx * 2 + i, ty * 2 + j) for j in range(2) for i in range(2)]
        for s in range(n):
            x, y = px[s % 4]
            ring.insert(*_single(x + 0.5, y + 0.5, 0.5, (0.5, 0.5, 0.5)))
    g = oracle.gradients(ring)
    st = oracle.tile_feedback(ring, g, S=2, m=2.0)
    for tile, n, empty, u in rows:
        assert st[int(tile), 0] == n and st[int(tile), 1] == empty
        assert abs(st[int(tile), 7] - u) < 1e-12


def test_tile_index_and_mean_gradients():
    """Tiles are row-major over a ceil(H/S) x ceil(W/S) grid, clipped at the
    border; the mean gradients average over the tile's non-empty pixels."""
    W, H, S = 5, 3, 2
    ring = oracle.Ring(W, H, 2)
    ring.insert(*_single(4.5, 2.5, 0.5, (1, 1, 1)))      # pixel (4,2) -> tile 5
    ring.insert(*_single(0.5, 0.5, 0.5, (1, 1, 1)))      # pixel (0,0) -> tile 0
    ring.insert(*_single(1.5, 0.5, 0.5, (0, 0, 0)))      # pixel (1,0) -> tile 0
    g = oracle.gradients(ring)
    st = oracle.tile_feedback(ring, g, S=S)
    assert st.shape[0] == 6
    np.testing.assert_array_equal(st[:, 0], [2, 0, 0, 0, 0, 1])
    np.testing.assert_array_equal(st[:, 1], [6, 8, 4, 4, 4, 1])
    # pixel (0,0) and (1,0) each see |1-0| on their one non-empty side
    np.testing.assert_allclose(st[0, 4], 1.0)


# --------------------------------------------------------------------------- reproject
def test_reproject_matches_float32_model_and_sorts_by_seq():
    rng = np.random.default_rng(3)
    W, H, b = 11, 7, 3
    ring = oracle.Ring(W, H, b)
    for _ in range(3):
        ring.insert(*_batch(rng, 150, W, H, t_sorted=False))
    t_now = np.float32(1.0)
    off, rec, rseq, dropped = oracle.reproject(ring, float(t_now))
    ent = []
    drop = 0
    for p in range(W * H):
        for k in range(ring.count[p]):
            s = ring.slot[p, k]
            a = np.float32(t_now - s[2])
            xp = np.float32(s[0] + np.float32(s[7] * a))
            yp = np.float32(s[1] + np.float32(s[8] * a))
            if not (0 <= xp < W and 0 <= yp < H):
                drop += 1
                continue
            q = int(math.floor(yp)) * W + int(math.floor(xp))
            ent.append((q, int(ring.seq[p, k]), xp, yp, s[2], s[4], s[5], s[6]))
    ent.sort(key=lambda e: (e[0], e[1]))
    assert dropped == drop and len(ent) == rec.shape[0]
    for i, e in enumerate(ent):
        assert rseq[i] == e[1]
        assert off[e[0]] <= i < off[e[0] + 1]
        np.testing.assert_array_equal(rec[i], np.array(e[2:], np.float32))


def test_pure_translation_is_exact():
    """Section 6.2: a point p0 moving at v, sampled at time t at p0 + v t,
    reprojects to p0 + v at t_now = 1 (up to float32 rounding)."""
    rng = np.random.default_rng(5)
    W = H = 64
    ring = oracle.Ring(W, H, 16)
    p0 = np.array([20.25, 30.75])
    v = np.array([12.5, -7.25])
    ts = np.sort(rng.uniform(0, 1, 16)).astype(np.float32)
    for t in ts:
        x, y = p0 + v * float(t)
        ring.insert(*_single(x, y, float(t), (1, 0, 0), mo=tuple(v)))
    off, rec, _, dropped = oracle.reproject(ring, 1.0)
    assert dropped == 0 and rec.shape[0] == 16
    np.testing.assert_allclose(rec[:, 0], p0[0] + v[0], atol=4e-5)
    np.testing.assert_allclose(rec[:, 1], p0[1] + v[1], atol=4e-5)


# --------------------------------------------------------------------------- sigma
def test_extent_identities():
    """Section 5.1: e_x G_x = e_y G_y = e_t G_t and e_x e_y e_t = V_S; with one
    spatial extent, e_s^2 e_t = V_S and e_s G_s = e_t G_t."""
    rng = np.random.default_rng(1)
    W, H, S = 16, 16, 4
    count = np.zeros(W * H, np.int32)
    count[rng.integers(0, W * H, 40)] = 1
    gx, gy, gt = rng.uniform(1e-3, 0.2, (3, W * H))
    theta = np.array([1.0, 0.0, 1e9, 1.0, 0.0, 1e9])
    ss, st = oracle.sigma(count, W, H, (None, gx, gy, gt), theta, S=S)
    # volumes from hand-counted tiles
    V = np.zeros(W * H)
    for y in range(H):
        for x in range(W):
            blk = count.reshape(H, W)[y // S * S:(y // S + 1) * S, x // S * S:(x // S + 1) * S]
            V[y * W + x] = S * S / blk.sum() if blk.sum() else S * S
    ok = (ss > 0.5) & (st > 0.05)
    assert ok.mean() > 0.5
    Gs = 0.5 * (gx + gy)
    np.testing.assert_allclose((ss * ss * st)[ok], V[ok], rtol=1e-12)
    np.testing.assert_allclose((ss * Gs)[ok], (st * gt)[ok], rtol=1e-12)


def test_sigma_closed_forms_and_clamps():
    W = H = 4
    count = np.full(W * H, 2, np.int32)        # V_S = 16 / 32 = 0.5 per 4x4 tile
    g = np.full(W * H, 0.1)
    ss, st = oracle.sigma(count, W, H, (None, g, g, g), np.array([1.0, 0, 1e9, 1.0, 0, 1e9]), S=4)
    np.testing.assert_allclose(ss, 0.5 ** (1 / 3), rtol=1e-12)   # G_s = G_t -> e = cbrt(V)
    np.testing.assert_allclose(st, 0.5 ** (1 / 3), rtol=1e-12)
    # static region: no temporal change -> long temporal, narrow spatial filter
    ss, st = oracle.sigma(count, W, H, (None, g, g, np.zeros(W * H)), oracle.DEFAULT_THETA, S=4)
    np.testing.assert_allclose(ss, 0.5)   # lower bound
    np.testing.assert_allclose(st, 1.0)   # upper clamp c_t
    # moving region: large temporal gradient, flat in space -> the reverse
    ss, st = oracle.sigma(count, W, H, (None, 0 * g, 0 * g, g * 50), oracle.DEFAULT_THETA, S=4)
    np.testing.assert_allclose(ss, 3.0)
    np.testing.assert_allclose(st, 0.05)
    # scale and offset
    th = np.array([2.0, 0.25, 1e9, 0.5, 0.125, 1e9])
    ss, st = oracle.sigma(count, W, H, (None, g, g, g), th, S=4)
    np.testing.assert_allclose(ss, 2.0 * 0.5 ** (1 / 3) + 0.25, rtol=1e-12)
    np.testing.assert_allclose(st, 0.5 * 0.5 ** (1 / 3) + 0.125, rtol=1e-12)


# --------------------------------------------------------------------------- filter
def _random_frame(rng, W, H, n, t_lo=0.0):
    rec = np.zeros((n, 6), np.float32)
    rec[:, 0] = rng.uniform(0, W, n)
    rec[:, 1] = rng.uniform(0, H, n)
    rec[:, 2] = rng.uniform(t_lo, 1, n)
    rec[:, 3:6] = rng.uniform(0, 1, (n, 3))
    q = np.floor(rec[:, 1]).astype(np.int64) * W + np.floor(rec[:, 0]).astype(np.int64)
    order = np.argsort(q, kind="stable")
    rec = rec[order]
    off = np.zeros(W * H + 1, np.uint32)
    np.add.at(off, q[order] + 1, 1)
    return np.cumsum(off).astype(np.uint32), rec


def test_filter_constant_colour_and_partition_of_unity():
    rng = np.random.default_rng(2)
    W, H = 12, 9
    off, rec = _random_frame(rng, W, H, 300)
    ss = rng.uniform(0.5, 3.0, W * H)
    st = rng.uniform(0.05, 1.0, W * H)
    rec[:, 3:6] = (0.25, 0.5, 1.0)
    out = oracle.filter_image(W, H, off, rec, ss, st)
    has = out[:, 3] > 0
    assert has.mean() > 0.9
    np.testing.assert_allclose(out[has, :3], np.broadcast_to([0.25, 0.5, 1.0], (has.sum(), 3)),
                               rtol=1e-12)
    rec[:, 3:6] = 1.0      # a channel of ones reconstructs to one: weights normalise
    out = oracle.filter_image(W, H, off, rec, ss, st)
    np.testing.assert_allclose(out[has, :3], 1.0, rtol=1e-12)


def test_filter_single_and_two_sample_closed_forms():
    W = H = 9
    R = 4
    ss = np.full(W * H, 1.3)
    st = np.full(W * H, 0.4)
    s1 = np.array([[4.3, 4.6, 0.5, 0.2, 0.4, 0.6]], np.float32)
    off = np.zeros(W * H + 1, np.uint32)
    off[4 * W + 4 + 1:] = 1
    out = oracle.filter_image(W, H, off, s1, ss, st, R=R)
    for j in range(H):
        for i in range(W):
            p = j * W + i
            if (i - 4) ** 2 + (j - 4) ** 2 <= R * R:
                d2 = (float(s1[0, 0]) - i - 0.5) ** 2 + (float(s1[0, 1]) - j - 0.5) ** 2
                w = math.exp(-d2 / (2 * 1.3 ** 2) - 0.5 ** 2 / (2 * 0.4 ** 2))
                np.testing.assert_allclose(out[p, :3], s1[0, 3:6], rtol=1e-7)
                assert abs(out[p, 3] - w) < 1e-12 * max(w, 1e-300)
            else:
                assert np.all(out[p] == 0.0)
    # two samples in different bins
    s2 = np.array([[2.2, 2.9, 0.9, 1.0, 0.0, 0.0], [5.7, 4.1, 0.1, 0.0, 0.0, 1.0]], np.float32)
    off = np.zeros(W * H + 1, np.uint32)
    off[2 * W + 2 + 1:] += 1
    off[4 * W + 5 + 1:] += 1
    out = oracle.filter_image(W, H, off, s2, ss, st, R=R)
    p = 3 * W + 4
    ws = []
    for s in s2:
        d2 = (float(s[0]) - 4.5) ** 2 + (float(s[1]) - 3.5) ** 2
        ws.append(math.exp(-d2 / (2 * 1.3 ** 2) - (1 - float(s[2])) ** 2 / (2 * 0.4 ** 2)))
    np.testing.assert_allclose(out[p, 0], ws[0] / (ws[0] + ws[1]), rtol=1e-12)
    np.testing.assert_allclose(out[p, 2], ws[1] / (ws[0] + ws[1]), rtol=1e-12)


@pytest.mark.parametrize("R", [2, 4])
def test_filter_binned_equals_brute_force_and_scatter(R):
    """The binned gather over the integer disc equals an all-samples-times-all-
    pixels loop and a sample-order (scatter) sum written in numpy: the filter
    shape is read at the pixel, so gather and scatter agree (section 5.2)."""
    rng = np.random.default_rng(R)
    W, H = 14, 11
    off, rec = _random_frame(rng, W, H, 500)
    ss = rng.uniform(0.5, 3.0, W * H)
    st = rng.uniform(0.05, 1.0, W * H)
    out = oracle.filter_image(W, H, off, rec, ss, st, R=R)
    brute = oracle.filter_brute(W, H, rec, ss, st, R=R)
    np.testing.assert_allclose(out, brute, rtol=1e-12, atol=1e-300)
    acc = np.zeros((W * H, 4))
    for s in rec.astype(np.float64):
        qi, qj = int(math.floor(s[0])), int(math.floor(s[1]))
        for dj in range(-R, R + 1):
            for di in range(-R, R + 1):
                i, j = qi + di, qj + dj
                if di * di + dj * dj > R * R or not (0 <= i < W and 0 <= j < H):
                    continue
                p = j * W + i
                d2 = (s[0] - i - 0.5) ** 2 + (s[1] - j - 0.5) ** 2
                w = math.exp(-d2 / (2 * ss[p] ** 2) - (1 - s[2]) ** 2 / (2 * st[p] ** 2))
                acc[p, :3] += w * s[3:6]
                acc[p, 3] += w
    nz = acc[:, 3] > 0
    np.testing.assert_allclose(out[nz, :3], acc[nz, :3] / acc[nz, 3:4], rtol=1e-10)
    np.testing.assert_allclose(out[:, 3], acc[:, 3], rtol=1e-10)


def test_static_region_weights_old_samples_moving_region_recent():
    """Sections 3 and 5.1: where the scene is static the temporal filter is
    broad and old samples keep weight; where it moves the filter is narrow
    and recent samples dominate. A 32x16 image: left half static, right half
    changes colour over time."""
    W, H, S = 32, 16, 16
    rng = np.random.default_rng(7)
    ring = oracle.Ring(W, H, 8)
    n = W * H * 8
    x = rng.uniform(0, W, n)
    y = rng.uniform(0, H, n)
    t = np.sort(rng.uniform(0, 1, n))
    pos = np.stack([x, y, t, np.full(n, 0.5)], 1).astype(np.float32)
    col = np.zeros((n, 4), np.float32)
    moving = x >= W / 2
    col[:, :3] = np.where(moving, t, 0.5)[:, None]          # right half brightens over time
    ring.insert(pos, col, np.zeros((n, 2), np.float32))
    res = oracle.reconstruct(ring, S=S)
    st = res["sig_t"].reshape(H, W)
    # (a pixel holding a single sample has no temporal gradient, so compare
    # typical widths rather than extremes)
    assert np.median(st[:, : W // 2 - 5]) > 3 * np.median(st[:, W // 2 + 5:])
    # share of weight carried by samples older than half a window at a pixel
    # in each half
    off, rec = res["off"], res["rec"]
    old = rec.copy()
    old[:, 3:6] = (rec[:, 2] < 0.5)[:, None]
    share = oracle.filter_image(W, H, off, old, res["sig_s"], res["sig_t"])[:, 0].reshape(H, W)
    static, moving = share[4:12, 4:10].mean(), share[4:12, 22:28].mean()
    assert static > 0.15 and moving < 0.05 and static > 5 * moving


# --------------------------------------------------------------------------- adjoint
def _loss(W, H, count, grads, off, rec, g, theta):
    ss, st = oracle.sigma(count, W, H, grads, theta)
    out = oracle.filter_image(W, H, off, rec, ss, st)
    return float((out[:, :3] * g).sum())


def test_backward_matches_central_differences():
    rng = np.random.default_rng(11)
    W, H = 20, 18
    ring = oracle.Ring(W, H, 4)
    pos, col, mo = _batch(rng, W * H * 3, W, H)
    ring.insert(pos, col, mo)
    grads = oracle.gradients(ring)
    off, rec, _, _ = oracle.reproject(ring)
    theta = np.array([0.9, 0.15, 2.4, 1.1, 0.02, 0.7])
    g = rng.normal(size=(W * H, 3))
    gcol, gth = oracle.backward(ring.count, W, H, grads, off, rec, g, theta)
    h = 1e-6
    for k in range(6):
        tp, tm = theta.copy(), theta.copy()
        tp[k] += h
        tm[k] -= h
        fd = (_loss(W, H, ring.count, grads, off, rec, g, tp)
              - _loss(W, H, ring.count, grads, off, rec, g, tm)) / (2 * h)
        assert abs(fd - gth[k]) <= 1e-5 * max(1.0, abs(fd)), (k, fd, gth[k])
    # colours: the loss is linear in each colour, so the difference is exact
    for e in rng.choice(rec.shape[0], 12, replace=False):
        for ch in range(3):
            rp, rm = rec.copy(), rec.copy()
            rp[e, 3 + ch] += 0.25
            rm[e, 3 + ch] -= 0.25
            fd = (_loss(W, H, ring.count, grads, off, rp, g, theta)
                  - _loss(W, H, ring.count, grads, off, rm, g, theta)) / 0.5
            hh = float(np.float32(rec[e, 3 + ch] + 0.25)) - float(np.float32(rec[e, 3 + ch] - 0.25))
            fd = fd * 0.5 / hh
            assert abs(fd - gcol[e, ch]) <= 1e-7 * max(1.0, abs(fd))


# ---- section 6.2: coverage-driven footprint sizes ------------------------------

def test_coverage_update_hand_cases():
    """Growth by 4 below 4 samples, shrinkage by 0.7 above 32, unchanged in
    between and without information, clamps, and the rounding to a disc."""
    W, H = 4, 1
    r = np.full(W * H, 2.0, np.float32)
    n = np.array([-1, 2, 10, 40], np.int32)
    r_next, R_next = oracle.coverage_update(W, H, r, n)
    assert r_next.tolist() == [2.0, 8.0, 2.0, float(np.float32(np.float32(2.0) * np.float32(0.7)))]
    assert R_next.tolist() == [2, 8, 2, 1]
    # boundaries: exactly 4 and exactly 32 samples change nothing
    r_next, _ = oracle.coverage_update(2, 1, np.full(2, 3.0, np.float32), np.array([4, 32], np.int32))
    assert r_next.tolist() == [3.0, 3.0]
    # clamps: growth stops at r_max, shrinkage at r_min; r = 2.5 rounds up
    r_next, R_next = oracle.coverage_update(3, 1, np.array([5.0, 5.0, 5.0], np.float32),
                                            np.array([0, 100, 5], np.int32), r_min=0.5, r_max=8.0)
    assert r_next.tolist()[0] == 8.0 and R_next[0] == 8
    r_next, R_next = oracle.coverage_update(1, 1, np.array([0.6], np.float32), np.array([100], np.int32))
    assert r_next[0] == np.float32(0.5) and R_next[0] == 1
    _, R_next = oracle.coverage_update(1, 1, np.array([2.5], np.float32), np.array([10], np.int32))
    assert R_next[0] == 3


def test_coverage_update_region_mean_at_borders():
    """The size is the mean over the pixel's 3x3 neighbourhood, clipped at the
    border (a corner averages 4 pixels, an edge 6, the interior 9)."""
    W, H = 3, 3
    r = np.arange(1, 10, dtype=np.float32)            # 1..9 row-major
    r_next, _ = oracle.coverage_update(W, H, r, np.full(9, 10, np.int32), r_max=100.0)
    g = r.reshape(3, 3).astype(np.float64)
    for j in range(3):
        for i in range(3):
            win = g[max(0, j - 1):j + 2, max(0, i - 1):i + 2]
            assert abs(r_next[j * 3 + i] - win.mean()) < 1e-6
    assert r_next[4] == np.float32(5.0)               # (1 + ... + 9) / 9


def test_coverage_count_matches_numpy():
    rng = np.random.default_rng(11)
    W, H = 13, 9
    off, rec = _random_frame(rng, W, H, 400)
    Rp = rng.integers(0, 5, W * H).astype(np.int32)
    n = oracle.coverage_count(W, H, Rp, off)
    cnt = np.diff(off.astype(np.int64)).reshape(H, W)
    for j in range(H):
        for i in range(W):
            R = Rp[j * W + i]
            ref = sum(int(cnt[j + dj, i + di]) for dj in range(-R, R + 1) for di in range(-R, R + 1)
                      if di * di + dj * dj <= R * R and 0 <= i + di < W and 0 <= j + dj < H)
            assert n[j * W + i] == ref


def test_per_pixel_radius_filter_equals_brute_force_and_fixed_radius():
    rng = np.random.default_rng(12)
    W, H = 12, 10
    off, rec = _random_frame(rng, W, H, 450)
    ss = rng.uniform(0.5, 3.0, W * H)
    st = rng.uniform(0.05, 1.0, W * H)
    Rp = rng.integers(0, 6, W * H).astype(np.int32)
    out = oracle.filter_image(W, H, off, rec, ss, st, R=Rp)
    brute = oracle.filter_brute(W, H, rec, ss, st, R=Rp)
    np.testing.assert_allclose(out, brute, rtol=1e-12, atol=1e-300)
    for R in (0, 3):
        fixed = oracle.filter_image(W, H, off, rec, ss, st, R=R)
        var = oracle.filter_image(W, H, off, rec, ss, st, R=np.full(W * H, R, np.int32))
        np.testing.assert_array_equal(fixed, var)


def test_coverage_fills_a_disocclusion_hole():
    """A region without samples is a hole at a small footprint; the next
    image grows the footprints there fourfold and fills it."""
    rng = np.random.default_rng(13)
    W, H, b = 24, 24, 4
    n = W * H * b
    pos = np.zeros((n, 4), np.float32)
    pos[:, 0] = rng.uniform(0, W, n)
    pos[:, 1] = rng.uniform(0, H, n)
    pos[:, 2] = np.sort(rng.uniform(0, 1, n))
    keep = (pos[:, 0] - 12) ** 2 + (pos[:, 1] - 12) ** 2 > 3.5 ** 2   # a hole of radius 3.5
    pos = pos[keep]
    col = np.zeros((len(pos), 4), np.float32)
    col[:, :3] = 0.5
    ring = oracle.Ring(W, H, b)
    ring.insert(pos, col, np.zeros((len(pos), 2), np.float32))
    state = {"r": np.full(W * H, 1.0, np.float32), "n": np.full(W * H, -1, np.int32)}
    first = oracle.reconstruct_adaptive(ring, state)
    holes = first["image"][:, 3] == 0
    assert holes.sum() > 0 and (first["R"] == 1).all()
    assert (state["n"][holes] < 4).all()
    second = oracle.reconstruct_adaptive(ring, state)
    assert (second["R"][holes] == 4).all()
    assert (second["image"][:, 3] > 0).all()
    np.testing.assert_allclose(second["image"][:, :3], 0.5, rtol=1e-12)


# ---- sections 6.1 and 4.1: tile error and gain control ------------------------

def test_tile_error_hand_example():
    """Two 2x2 tiles, b = 2: E = s (kappa v / sum v + lambda u / sum u +
    (1 - kappa - lambda) o / sum o) with o = occluded / (s b), worked by hand."""
    ring = oracle.Ring(4, 2, 2)                       # empty: the records below are given
    tiles = np.zeros((2, oracle.NT))
    tiles[:, 3] = [1.0, 3.0]                          # variance of luminance
    tiles[:, 7] = [0.5, 0.0]                          # undersampling u
    E, _ = oracle.tile_error(ring, tiles, S=2, occluded=[2.0, 6.0], kappa=0.5, lam=0.3)
    np.testing.assert_allclose(E, [4 * (0.5 * 0.25 + 0.3 * 1.0 + 0.2 * 0.25),
                                   4 * (0.5 * 0.75 + 0.0 + 0.2 * 0.75)], rtol=1e-14)
    # without occlusion data, or with all-zero sums, a term adds nothing
    E, _ = oracle.tile_error(ring, tiles, S=2, kappa=0.5, lam=0.3)
    np.testing.assert_allclose(E, [4 * (0.125 + 0.3), 4 * 0.375], rtol=1e-14)
    tiles[:, 7] = 0.0
    E, _ = oracle.tile_error(ring, tiles, S=2, kappa=0.5, lam=0.3)
    np.testing.assert_allclose(E, [0.5, 1.5], rtol=1e-14)


def test_tile_error_shares_sum_to_the_weights():
    """Each term is a share of a sum over tiles: sum_t E_t / s_t = kappa +
    lambda + (1 - kappa - lambda) whenever every sum is positive."""
    rng = np.random.default_rng(21)
    W, H, b = 70, 45, 4
    pos, col, mo = _batch(rng, W * H * 8, W, H)
    keep = (pos[:, 0] < 48) | (pos[:, 1] < 16) | (rng.uniform(0, 1, len(pos)) < 0.05)   # a sparse corner
    pos, col, mo = pos[keep], col[keep], mo[keep]
    ring = oracle.Ring(W, H, b)
    ring.insert(pos, col, mo)
    grads = oracle.gradients(ring)
    tiles = oracle.tile_feedback(ring, grads, S=16)
    occ = rng.integers(0, 5, tiles.shape[0]).astype(np.float64)
    E, _ = oracle.tile_error(ring, tiles, S=16, occluded=occ, kappa=0.3, lam=0.45)
    ntx = -(-W // 16)
    A = np.array([min(16, W - (t % ntx) * 16) * min(16, H - (t // ntx) * 16) for t in range(len(E))])
    assert (tiles[:, 7] > 0).any() and tiles[:, 3].sum() > 0
    np.testing.assert_allclose((E / A).sum(), 1.0, rtol=1e-12)


def test_gain_control_on_a_ramp_in_space_and_time():
    """Grey colour a x + c t at pixel centres, sampled at t = 0.25 and 0.75:
    G_x = a, G_y = 0, G_t = c everywhere, every sample age is 0.75 or 0.25, so
    dC/ds = a / 2, dC/dt = c, T = 0.5 and S* = i c T / (a / 2)."""
    a, c, i = 0.02, 0.3, 1.5
    W, H = 40, 24
    ring = _grid_ring(W, H, 4, lambda x, y, t: (a * x + c * t,) * 3)
    grads = oracle.gradients(ring)
    tiles = oracle.tile_feedback(ring, grads, S=8)
    _, gain = oracle.tile_error(ring, tiles, S=8, importance=i)
    dcds, dcdt, T, Sw, N = gain
    np.testing.assert_allclose([dcds, dcdt, T], [a / 2, c, 0.5], rtol=1e-5)
    np.testing.assert_allclose(Sw, i * c * 0.5 / (a / 2), rtol=1e-5)
    np.testing.assert_allclose(N, max(1.0, W * H / Sw ** 2), rtol=1e-5)


# ---- section 5.2: the reconstructor's global FIFO buffer ---------------------------

def test_fifo_keeps_the_n_most_recent_accepted_samples():
    rng = np.random.default_rng(31)
    W, H, N = 9, 7, 37
    fifo = oracle.Fifo(W, H, N)
    model = collections.deque(maxlen=N)
    seq = 0
    for n in (20, 31, 5, 60):
        pos, col, mo = _batch(rng, n, W, H, bad_frac=0.2)
        rej = fifo.insert(pos, col, mo)
        bad = 0
        for i in range(n):
            x, y, t = pos[i, 0], pos[i, 1], pos[i, 2]
            vals = [x, y, t, col[i, 0], col[i, 1], col[i, 2], mo[i, 0], mo[i, 1]]
            if not all(np.isfinite(vals)) or not (0 <= x < W and 0 <= y < H):
                bad += 1
                continue
            model.append((seq + i, [x, y, t, pos[i, 3], col[i, 0], col[i, 1], col[i, 2], mo[i, 0], mo[i, 1]]))
        seq += n
        assert rej == bad
        k = fifo.resident
        assert k == len(model)
        got = sorted(zip(fifo.seq[:k].tolist(), fifo.q[:k].tolist()))
        want = [(s, list(np.float32(v))) for s, v in model]
        assert [s for s, _ in got] == [s for s, _ in want]
        np.testing.assert_array_equal(np.array([v for _, v in got], np.float32),
                                      np.array([v for _, v in want], np.float32))


def test_fifo_frame_view_matches_float32_model():
    """The FIFO's frame view: every sample moved in single precision with one
    rounding per operation, off-image ones dropped, the rest ordered by bin
    and sequence number."""
    rng = np.random.default_rng(32)
    W, H, N = 17, 12, 300
    fifo = oracle.Fifo(W, H, N)
    for n in (250, 180):
        fifo.insert(*_batch(rng, n, W, H))
    off, rec, rseq, dropped = oracle.reproject_fifo(fifo, 1.0)
    k = fifo.resident
    q, sq = fifo.q[:k], fifo.seq[:k]
    a = np.float32(1.0) - q[:, 2]
    xp = q[:, 0] + q[:, 7] * a
    yp = q[:, 1] + q[:, 8] * a
    ok = (xp >= 0) & (xp < W) & (yp >= 0) & (yp < H)
    assert dropped == int((~ok).sum())
    bins = np.floor(yp[ok]).astype(np.int64) * W + np.floor(xp[ok]).astype(np.int64)
    order = np.lexsort((sq[ok], bins))
    np.testing.assert_array_equal(rseq, sq[ok][order])
    np.testing.assert_array_equal(rec[:, 0], xp[ok][order])
    np.testing.assert_array_equal(rec[:, 1], yp[ok][order])
    np.testing.assert_array_equal(rec[:, 3:6], q[ok][order][:, 4:7])
    np.testing.assert_array_equal(np.diff(off.astype(np.int64)), np.bincount(bins, minlength=W * H))


# ---- section 6.2 with camera matrices ---------------------------------------------

def _camera_ring(rng, W, H, b, n, grid=64.0):
    """Samples whose stored hit points lie on a 1/grid lattice, so that the
    screen mappings below are exact in single precision."""
    ring = oracle.Ring(W, H, b)
    X = np.floor(rng.uniform(0, W, n) * grid) / grid
    Y = np.floor(rng.uniform(0, H, n) * grid) / grid
    t = np.sort(rng.uniform(0, 1, n)).astype(np.float32)
    pos = np.stack([X, Y, t, rng.uniform(0, 1, n)], 1).astype(np.float32)
    col = np.zeros((n, 4), np.float32)
    col[:, :3] = rng.uniform(0, 1, (n, 3))
    ring.insert(pos, col, np.zeros((n, 2), np.float32))
    world = np.stack([X, Y, rng.uniform(1, 5, n), np.zeros(n)], 1).astype(np.float32)
    return ring, world


def _screen_camera(W, H, dx=0.0, dy=0.0):
    """World (X, Y) in pixels to NDC, the camera moved by (dx, dy) pixels."""
    return np.array([[2 / W, 0, 0, -1 - 2 * dx / W], [0, 2 / H, 0, -1 - 2 * dy / H], [0, 0, 1, 0], [0, 0, 0, 1]],
                    np.float32)


def test_camera_identity_and_pan_are_exact():
    rng = np.random.default_rng(41)
    W, H, b = 64, 32, 4
    ring, world = _camera_ring(rng, W, H, b, 700)
    off, rec, rseq, dropped = oracle.reproject_camera(ring, world, _screen_camera(W, H))
    assert dropped == 0
    np.testing.assert_array_equal(rec[:, 0], world[rseq, 0])
    np.testing.assert_array_equal(rec[:, 1], world[rseq, 1])
    off2, rec2, rseq2, dropped2 = oracle.reproject_camera(ring, world, _screen_camera(W, H, dx=4.0, dy=-2.0))
    keep = (world[rseq, 0] - 4 >= 0) & (world[rseq, 1] + 2 < H)
    assert dropped2 == int((~keep).sum())
    want = np.stack([world[:, 0] - 4, world[:, 1] + 2], 1)
    np.testing.assert_array_equal(rec2[:, :2], want[rseq2])


def test_camera_projection_matches_float32_model():
    rng = np.random.default_rng(42)
    W, H, b = 48, 40, 4
    n = 900
    ring = oracle.Ring(W, H, b)
    pos, col, mo = _batch(rng, n, W, H)
    ring.insert(pos, col, mo)
    world = np.stack([rng.uniform(-2, 2, n), rng.uniform(-2, 2, n), rng.uniform(2, 6, n), np.zeros(n)],
                     1).astype(np.float32)
    f = np.float32
    vp = np.array([[1.2, 0.1, 0.05, 0.02], [-0.05, 1.3, 0.1, -0.1], [0, 0, 1, 0], [0.01, 0.02, 0.4, 0.3]], f)
    world[:7, 2] = -5.0                                    # behind the camera
    off, rec, rseq, dropped = oracle.reproject_camera(ring, world, vp, 1.0)
    count, slot, seq = ring.count, ring.slot, ring.seq
    rows = []
    for p in range(W * H):
        for k in range(count[p]):
            s, q = slot[p, k], seq[p, k]
            w = world[q]
            c = [f(f(f(vp[r, 0] * w[0]) + f(vp[r, 1] * w[1])) + f(vp[r, 2] * w[2])) + vp[r, 3] for r in (0, 1, 3)]
            if not c[2] > 0:
                continue
            a = f(f(1.0) - s[2])
            xp = f(f(f(f(c[0] / c[2]) * f(0.5)) + f(0.5)) * f(W)) + f(s[7] * a)
            yp = f(f(f(f(c[1] / c[2]) * f(0.5)) + f(0.5)) * f(H)) + f(s[8] * a)
            if 0 <= xp < W and 0 <= yp < H:
                rows.append((int(np.floor(yp)) * W + int(np.floor(xp)), int(q), xp, yp))
    rows.sort(key=lambda r: (r[0], r[1]))
    assert dropped == ring.resident - len(rows)
    np.testing.assert_array_equal(rseq, [r[1] for r in rows])
    np.testing.assert_array_equal(rec[:, 0], np.array([r[2] for r in rows], np.float32))
    np.testing.assert_array_equal(rec[:, 1], np.array([r[3] for r in rows], np.float32))

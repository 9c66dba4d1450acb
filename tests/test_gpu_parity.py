"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer work (queues, eviction, frame bins, order, tile counts) must match
bit for bit. Floating point follows FP32-vs-FP64 tolerances per stage; each
stage is checked on the oracle's own input to that stage (imported through
the ABI) so that the tolerance measures that stage's arithmetic alone:

* gradients:  |d| <= 1e-5 |ref| + 2e-8 (the luminances and their weighted
              means are double-float; the age weights are FP32, whose relative
              error ~1e-7 times the spread of a pixel's luminances bounds the
              absolute error of the spatial gradients, a difference of means)
* widths:     relative 1e-5
* filter:     relative 1e-5 per channel with denominator max(|ref|, 1e-3)
"""
import math

import numpy as np
import pytest
import torch

import oracle
from workloads import scenes

pytestmark = pytest.mark.gpu

from paper_2510_15876_gb300 import _lib as L  # noqa: E402

T_NOW = 1.0


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_15876_gb300.build import build
    build()
    return torch.device("cuda:0")


def _mk(dev, W, H, b, ct="f32", **kw):
    from paper_2510_15876_gb300.api import Reconstructor
    return Reconstructor(W, H, b, color_type=ct, device=dev, **kw)


def _upload(rec, batch, dtype=torch.float32):
    from paper_2510_15876_gb300.api import to_device_batch
    pos, col, mo = to_device_batch(batch, rec.device, dtype)
    rec.insert(pos, col, mo)
    torch.cuda.synchronize()


def _scene_batch(key, seed=0, n=None, W=None, H=None, b=None, speed=None, discs=None):
    spec = scenes.CONFIGS[key]
    if W is not None:
        import dataclasses
        spec = dataclasses.replace(spec, key=f"{key}-{W}x{H}x{b}", width=W, height=H, depth=b,
                                   speed=spec.speed if speed is None else speed,
                                   n_discs=spec.n_discs if discs is None else discs, edge_fraction=None,
                                   importance=False)
    sc = scenes.make_scene(spec, seed)
    return sc, scenes.sample_stream(sc, n if n is not None else spec.n_samples, seed)


def _random_batch(rng, n, W, H, bad=0.0):
    x = rng.uniform(0, W, n).astype(np.float32)
    y = rng.uniform(0, H, n).astype(np.float32)
    t = np.sort(rng.uniform(0, 1, n)).astype(np.float32)
    pos = np.stack([x, y, t, rng.uniform(0, 1, n).astype(np.float32)], 1)
    col = np.zeros((n, 4), np.float32)
    col[:, :3] = rng.uniform(0, 1, (n, 3))
    mo = rng.uniform(-4, 4, (n, 2)).astype(np.float32)
    if bad:
        k = int(n * bad)
        idx = rng.choice(n, k, replace=False)
        pos[idx[0::4], 0] = np.nan
        pos[idx[1::4], 0] = W
        col[idx[2::4], 2] = np.inf
        mo[idx[3::4], 1] = -np.inf
    return {"pos": pos, "color": col, "motion": mo}


def _ring_equal(rec, ring):
    count, slot, seq = rec.export_ring()
    np.testing.assert_array_equal(count, ring.count)
    np.testing.assert_array_equal(seq, ring.seq)
    np.testing.assert_array_equal(slot, ring.slot)


def _grad_close(got, want):
    ok = np.isnan(want) == np.isnan(got)
    assert ok.all()
    m = ~np.isnan(want)
    err = np.abs(got[m] - want[m])
    bound = 1e-5 * np.abs(want[m]) + 2e-8
    assert (err <= bound).all(), f"max excess {np.max(err - bound):.3g}"


def _rel_err(got, want, floor=1e-3):
    return np.abs(got - want) / np.maximum(np.abs(want), floor)


# ----------------------------------------------------------------------------- ingest
@pytest.mark.parametrize("W,H,b,n,batches", [(7, 5, 1, 300, 3), (7, 5, 4, 2000, 2), (33, 17, 16, 4000, 3),
                                             (128, 128, 4, 65536, 1), (131, 67, 8, 30000, 4)])
def test_ingest_bitexact(dev, W, H, b, n, batches):
    """Queues, eviction order and sequence numbers match the oracle bit for bit,
    including pixels that receive more than 32 samples in one batch and
    batches with rejected samples."""
    rng = np.random.default_rng(W * 1000 + b)
    rec = _mk(dev, W, H, b)
    ring = oracle.Ring(W, H, b)
    for k in range(batches):
        batch = _random_batch(rng, n, W, H, bad=0.05 if k == 1 else 0.0)
        _upload(rec, batch)
        ring.insert(batch["pos"], batch["color"], batch["motion"])
    _ring_equal(rec, ring)
    info = rec.query()
    assert info["rejected"] == ring.rejected and info["resident"] == ring.resident
    assert info["inserted"] == ring.total


@pytest.mark.parametrize("W,H,b,dense,spread,batches", [(16, 8, 4, 0, 10000, 2), (40, 20, 8, 8000, 3000, 2),
                                                        (37, 19, 32, 0, 60000, 1), (10, 7, 16, 0, 50000, 2)])
def test_ingest_dense_tiles_bitexact(dev, W, H, b, dense, spread, batches):
    """Dense batches: tens of records a pixel (ranked by a thread per record,
    with pixels crossing the commit's shared-memory tiles), one pixel with
    8,000 records and every pixel of a 10 x 7 image above 256 records (a warp
    streams the pixel's bucket keeping its newest 32), rejected samples, over
    consecutive batches, bit for bit against the oracle's queues."""
    rng = np.random.default_rng(W + H + b)
    rec = _mk(dev, W, H, b)
    ring = oracle.Ring(W, H, b)
    for k in range(batches):
        batch = _random_batch(rng, dense + spread, W, H, bad=0.02)
        if dense:
            idx = rng.permutation(dense + spread)[:dense]
            batch["pos"][idx, 0] = 3.0 + rng.uniform(0, 0.99, dense).astype(np.float32)
            batch["pos"][idx, 1] = 2.5
        _upload(rec, batch)
        ring.insert(batch["pos"], batch["color"], batch["motion"])
    _ring_equal(rec, ring)
    info = rec.query()
    assert info["rejected"] == ring.rejected and info["resident"] == ring.resident


def test_ingest_scene_stream(dev):
    sc, batch = _scene_batch("c1_128x128x4")
    rec = _mk(dev, 128, 128, 4)
    ring = oracle.Ring(128, 128, 4)
    _upload(rec, batch)
    ring.insert(batch["pos"], batch["color"], batch["motion"])
    _ring_equal(rec, ring)


# ----------------------------------------------------------------------------- gradients + tiles
def _setup_scene(dev, W, H, b, seed=1, ct="f32", speed=24.0, discs=12, S=32, R=4):
    sc, batch = _scene_batch("c4_512x512x8", seed, W=W, H=H, b=b, speed=speed, discs=discs)
    rec = _mk(dev, W, H, b, ct=ct, tile=S, radius=R)
    ring = oracle.Ring(W, H, b)
    _upload(rec, batch, rec.color_dtype)
    col = batch["color"]
    if ct != "f32":
        col = torch.from_numpy(col).to(rec.color_dtype).float().numpy()
    ring.insert(batch["pos"], col, batch["motion"])
    return sc, batch, rec, ring


@pytest.mark.parametrize("W,H,b", [(128, 128, 4), (131, 67, 8), (96, 80, 16)])
def test_gradients_match_oracle(dev, W, H, b):
    _, _, rec, ring = _setup_scene(dev, W, H, b)
    rec.estimate_gradients(T_NOW)
    L_, gx, gy, gt = oracle.gradients(ring, T_NOW)
    _grad_close(rec.export_map(L.AFR_MAP_LBAR).astype(np.float64), L_)
    _grad_close(rec.export_map(L.AFR_MAP_GX).astype(np.float64), gx)
    _grad_close(rec.export_map(L.AFR_MAP_GY).astype(np.float64), gy)
    _grad_close(rec.export_map(L.AFR_MAP_GT).astype(np.float64), gt)


def test_temporal_gradient_out_of_time_order(dev):
    """Insertion order differing from time order: pairs follow time."""
    rng = np.random.default_rng(4)
    W, H, b = 16, 8, 8
    rec = _mk(dev, W, H, b)
    ring = oracle.Ring(W, H, b)
    for _ in range(3):
        batch = _random_batch(rng, 600, W, H)
        batch["pos"][:, 2] = rng.uniform(0, 1, 600).astype(np.float32)   # unsorted times
        _upload(rec, batch)
        ring.insert(batch["pos"], batch["color"], batch["motion"])
    rec.estimate_gradients(T_NOW)
    _, _, _, gt = oracle.gradients(ring, T_NOW)
    _grad_close(rec.export_map(L.AFR_MAP_GT).astype(np.float64), gt)


@pytest.mark.parametrize("W,H,b,S", [(128, 128, 4, 32), (131, 67, 8, 32), (100, 70, 16, 16)])
def test_tile_feedback_matches_oracle(dev, W, H, b, S):
    from paper_2510_15876_gb300.api import decode_tiles
    _, _, rec, ring = _setup_scene(dev, W, H, b, S=S)
    rec.estimate_gradients(T_NOW)
    got = decode_tiles(rec.tile_feedback())
    grads = oracle.gradients(ring, T_NOW)
    want = oracle.tile_feedback(ring, grads, S=S, t_now=T_NOW, m=2.0)
    np.testing.assert_array_equal(got["n"], want[:, 0].astype(np.uint32))
    np.testing.assert_array_equal(got["empty_slots"], want[:, 1].astype(np.uint32))
    np.testing.assert_allclose(got["mean_L"], want[:, 2], rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(got["var_L"], want[:, 3], rtol=1e-4, atol=1e-6)
    for k, f in ((4, "mean_Gx"), (5, "mean_Gy"), (6, "mean_Gt")):
        np.testing.assert_allclose(got[f], want[:, k], rtol=1e-4, atol=2e-6)
    np.testing.assert_allclose(got["u"], want[:, 7], rtol=1e-6, atol=1e-6)


# ----------------------------------------------------------------------------- reprojection
@pytest.mark.parametrize("W,H,b", [(128, 128, 4), (131, 67, 8), (64, 48, 16)])
def test_reproject_bitexact(dev, W, H, b):
    _, _, rec, ring = _setup_scene(dev, W, H, b, speed=48.0)
    rec.reproject(T_NOW)
    off, frec, fseq = rec.export_frame()
    woff, wrec, wseq, dropped = oracle.reproject(ring, T_NOW)
    np.testing.assert_array_equal(off, woff)
    np.testing.assert_array_equal(fseq, wseq)
    np.testing.assert_array_equal(frec[:, :2], wrec[:, :2])          # x', y' bit-exact
    np.testing.assert_array_equal(frec[:, 3:6], wrec[:, 3:6])
    a = (np.float32(T_NOW) - wrec[:, 2]).astype(np.float32)
    np.testing.assert_array_equal(frec[:, 2], (a * a).astype(np.float32))
    assert rec.query()["dropped"] == dropped
    assert rec.query()["unsorted_bins"] == 0


# ----------------------------------------------------------------------------- widths + filter
def _oracle_maps_f32(ring):
    L_, gx, gy, gt = oracle.gradients(ring, T_NOW)
    return tuple(np.nan_to_num(v, nan=np.nan).astype(np.float32) for v in (L_, gx, gy, gt))


@pytest.mark.parametrize("W,H,b", [(128, 128, 4), (131, 67, 8)])
def test_widths_match_oracle(dev, W, H, b):
    _, _, rec, ring = _setup_scene(dev, W, H, b)
    rec.estimate_gradients(T_NOW)
    rec.reproject(T_NOW)
    L32, gx, gy, gt = _oracle_maps_f32(ring)
    rec.import_map(L.AFR_MAP_GX, gx)
    rec.import_map(L.AFR_MAP_GY, gy)
    rec.import_map(L.AFR_MAP_GT, gt)
    theta = np.array([0.8, 0.1, 2.5, 1.2, 0.02, 0.9])
    rec.reconstruct(T_NOW, theta)
    ss, st = oracle.sigma(ring.count, W, H, (None, gx.astype(np.float64), gy.astype(np.float64),
                                            gt.astype(np.float64)), theta, S=32)
    np.testing.assert_allclose(rec.export_map(L.AFR_MAP_SIGMA_S), ss, rtol=1e-5)
    np.testing.assert_allclose(rec.export_map(L.AFR_MAP_SIGMA_T), st, rtol=1e-5)


def _filter_stage(dev, W, H, b, R=4, speed=24.0, seed=1):
    _, _, rec, ring = _setup_scene(dev, W, H, b, R=R, speed=speed, seed=seed)
    rec.estimate_gradients(T_NOW)
    rec.reproject(T_NOW)
    grads = oracle.gradients(ring, T_NOW)
    ss, st = oracle.sigma(ring.count, W, H, grads, oracle.DEFAULT_THETA)
    ss32, st32 = ss.astype(np.float32), st.astype(np.float32)
    rec.import_map(L.AFR_MAP_SIGMA_S, ss32)
    rec.import_map(L.AFR_MAP_SIGMA_T, st32)
    img = rec.reconstruct(T_NOW, flags=L.AFR_RECON_KEEP_SIGMA).cpu().numpy().reshape(-1, 4).astype(np.float64)
    off, frec, _, _ = oracle.reproject(ring, T_NOW)
    ref = oracle.filter_image(W, H, off, frec, ss32.astype(np.float64), st32.astype(np.float64), R=R)
    return img, ref


def _check_filter(img, ref, tol=1e-5):
    hole = ref[:, 3] == 0
    np.testing.assert_array_equal(img[hole], 0.0)
    # W is reported as S 2^-m in FP32: nonzero wherever the exact W is within
    # FP32's normal range (a pixel whose samples are all far older than its
    # temporal width may report W = 0 and still have exact colours)
    assert (img[ref[:, 3] > 1e-30, 3] > 0).all()
    err = _rel_err(img[~hole, :3], ref[~hole, :3])
    assert err.max() <= tol, f"max rel err {err.max():.3g} (p99.9 {np.quantile(err, 0.999):.3g})"
    big = ref[:, 3] > 1e-30
    np.testing.assert_allclose(img[big, 3], ref[big, 3], rtol=1e-4)


@pytest.mark.parametrize("W,H,b,R", [(128, 128, 4, 4), (131, 67, 8, 4), (96, 80, 16, 4), (64, 40, 8, 2),
                                     (48, 33, 4, 0), (40, 40, 8, 7)])
def test_filter_matches_oracle(dev, W, H, b, R):
    img, ref = _filter_stage(dev, W, H, b, R=R)
    _check_filter(img, ref)


def test_filter_old_samples_and_narrow_temporal_width(dev):
    """Every sample one window old with the narrowest temporal width: all
    weights are ~2^-29 per sample in float terms; the per-pixel exponent shift
    keeps the normalised colour exact."""
    W, H, b = 40, 30, 4
    rng = np.random.default_rng(9)
    batch = _random_batch(rng, W * H * b, W, H)
    batch["pos"][:, 2] = 0.0
    rec = _mk(dev, W, H, b)
    ring = oracle.Ring(W, H, b)
    _upload(rec, batch)
    ring.insert(batch["pos"], batch["color"], batch["motion"])
    rec.estimate_gradients(T_NOW)
    rec.reproject(T_NOW)
    ss = np.full(W * H, 0.5, np.float32)
    st = np.full(W * H, 0.05, np.float32)
    rec.import_map(L.AFR_MAP_SIGMA_S, ss)
    rec.import_map(L.AFR_MAP_SIGMA_T, st)
    img = rec.reconstruct(T_NOW, flags=L.AFR_RECON_KEEP_SIGMA).cpu().numpy().reshape(-1, 4).astype(np.float64)
    off, frec, _, _ = oracle.reproject(ring, T_NOW)
    ref = oracle.filter_image(W, H, off, frec, ss.astype(np.float64), st.astype(np.float64))
    hole = ref[:, 3] == 0
    err = _rel_err(img[~hole, :3], ref[~hole, :3])
    assert err.max() <= 1e-5


def test_filter_brute_force_tiny(dev):
    """On a tiny image the GPU equals the oracle's all-samples x all-pixels loop."""
    W, H, b = 13, 9, 4
    _, _, rec, ring = _setup_scene(dev, W, H, b, speed=6.0, discs=3)
    rec.estimate_gradients(T_NOW)
    rec.reproject(T_NOW)
    grads = oracle.gradients(ring, T_NOW)
    ss, st = oracle.sigma(ring.count, W, H, grads, oracle.DEFAULT_THETA)
    ss32, st32 = ss.astype(np.float32), st.astype(np.float32)
    rec.import_map(L.AFR_MAP_SIGMA_S, ss32)
    rec.import_map(L.AFR_MAP_SIGMA_T, st32)
    img = rec.reconstruct(T_NOW, flags=L.AFR_RECON_KEEP_SIGMA).cpu().numpy().reshape(-1, 4).astype(np.float64)
    _, frec, _, _ = oracle.reproject(ring, T_NOW)
    ref = oracle.filter_brute(W, H, frec, ss32.astype(np.float64), st32.astype(np.float64))
    _check_filter(img, ref)


def test_empty_buffer_is_all_holes(dev):
    rec = _mk(dev, 20, 10, 4)
    rec.estimate_gradients(T_NOW)
    rec.reproject(T_NOW)
    img = rec.reconstruct(T_NOW).cpu().numpy()
    assert (img == 0).all()
    assert rec.query()["frame"] == 0


def test_call_order_is_enforced(dev):
    rec = _mk(dev, 20, 10, 4)
    with pytest.raises(L.AfrError) as e:
        rec.reconstruct(T_NOW)
    assert e.value.status == L.AFR_ERR_BAD_STATE
    rec.estimate_gradients(T_NOW)
    rec.reproject(0.5)
    with pytest.raises(L.AfrError) as e:
        rec.reconstruct(T_NOW)
    assert e.value.status == L.AFR_ERR_BAD_STATE
    with pytest.raises(L.AfrError) as e:
        rec.backward(torch.zeros((10, 20, 4), device=dev))
    assert e.value.status == L.AFR_ERR_BAD_STATE
    assert rec.status() == L.AFR_OK


@pytest.mark.parametrize("W,H,b", [(96, 80, 4), (640, 360, 8)])
def test_refresh_matches_serial_calls(dev, W, H, b):
    """refresh() runs the gradient branch on a side stream beside the
    reprojection: the same image and tile statistics, bit for bit, as the
    calls in series, over several refreshes of a changing buffer."""
    sc, batch = _scene_batch("c4_512x512x8", seed=3, n=W * H * b, W=W, H=H, b=b)
    a, s = _mk(dev, W, H, b), _mk(dev, W, H, b)
    cuts = np.linspace(0, len(batch["pos"]), 4).astype(int)
    for i, (lo, hi) in enumerate(zip(cuts[:-1], cuts[1:])):
        part = {k: np.ascontiguousarray(v[lo:hi]) for k, v in batch.items()}
        _upload(a, part)
        _upload(s, part)
        t = T_NOW - 0.1 * (2 - i)
        img_a, tiles_a = a.refresh(t)
        s.estimate_gradients(t)
        s.reproject(t)
        img_s = s.reconstruct(t)
        tiles_s = s.tile_feedback()
        assert torch.equal(img_a, img_s) and torch.equal(tiles_a, tiles_s)
    assert a.query() == s.query()


def test_pipelined_steps_match_serial(dev):
    """The next batch's reset and insert on another stream, waiting only for
    refresh()'s reads_done event, overlap the current image's filter: every
    image and tile record equals the one from calls in series."""
    from paper_2510_15876_gb300.api import to_device_batch
    W, H, b = 640, 360, 8
    batches = []
    for seed in range(4):
        _, bt = _scene_batch("c4_512x512x8", seed=seed, n=W * H * b, W=W, H=H, b=b, speed=24.0 + 8 * seed)
        batches.append(to_device_batch(bt, dev))
    a, s = _mk(dev, W, H, b), _mk(dev, W, H, b)
    want = []
    for pos, col, mo in batches:
        s.reset()
        s.insert(pos, col, mo)
        s.estimate_gradients(T_NOW)
        s.reproject(T_NOW)
        want.append((s.reconstruct(T_NOW), s.tile_feedback()))
    main, ingest = torch.cuda.current_stream(), torch.cuda.Stream(dev)
    reads_done, ingested = torch.cuda.Event(), torch.cuda.Event()
    reads_done.record(main)
    got = []
    for pos, col, mo in batches:
        ingest.wait_event(reads_done)
        a.reset(stream=ingest)
        a.insert(pos, col, mo, stream=ingest)
        ingested.record(ingest)
        main.wait_event(ingested)
        got.append(a.refresh(T_NOW, reads_done=reads_done))
    torch.cuda.synchronize()
    for (img, tiles), (img_w, tiles_w) in zip(got, want):
        assert torch.equal(img, img_w) and torch.equal(tiles, tiles_w)


def test_pipelined_binning_matches_serial(dev):
    """afr_insert_samples_ex with the reset flag and refresh()'s reads_done
    event: the next batch's binning starts at once, beside the current
    image's gradients and reprojection, and only its reset and commit wait
    for the event. Every image, tile record and counter equals the calls in
    series; the buffers change every step and a batch carries rejected
    samples."""
    from paper_2510_15876_gb300.api import to_device_batch
    W, H, b = 640, 360, 8
    batches = []
    for seed in range(4):
        _, bt = _scene_batch("c4_512x512x8", seed=seed, n=W * H * b, W=W, H=H, b=b, speed=24.0 + 8 * seed)
        if seed == 2:
            bt["pos"][::97, 0] = np.nan
            bt["color"][5::89, 1] = np.inf
        batches.append(to_device_batch(bt, dev))
    a, s = _mk(dev, W, H, b), _mk(dev, W, H, b)
    want = []
    for pos, col, mo in batches:
        s.reset()
        s.insert(pos, col, mo)
        s.estimate_gradients(T_NOW)
        s.reproject(T_NOW)
        want.append((s.reconstruct(T_NOW), s.tile_feedback(), s.query()))
    main, ingest = torch.cuda.current_stream(), torch.cuda.Stream(dev)
    reads_done, ingested = torch.cuda.Event(), torch.cuda.Event()
    reads_done.record(main)
    got = []
    for pos, col, mo in batches:
        a.insert(pos, col, mo, stream=ingest, reset=True, queues_free=reads_done)
        ingested.record(ingest)
        main.wait_event(ingested)
        img, tiles = a.refresh(T_NOW, reads_done=reads_done)
        torch.cuda.synchronize()
        got.append((img.clone(), tiles.clone(), a.query()))
    for (img, tiles, q), (img_w, tiles_w, q_w) in zip(got, want):
        assert torch.equal(img, img_w) and torch.equal(tiles, tiles_w)
        assert q == q_w


@pytest.mark.parametrize("kind", ["queues", "fifo", "world"])
def test_insert_ex_equals_reset_and_insert(dev, kind):
    """afr_insert_samples_ex(AFR_INSERT_RESET, event recorded on another
    stream) leaves the per-pixel queues (or the reconstructor queue, or the
    hit points) exactly as afr_reset followed by afr_insert_samples, after a
    first batch filled them; unknown flags are refused."""
    from paper_2510_15876_gb300 import _lib as L
    W, H, b = 131, 67, 8
    rng = np.random.default_rng(7)
    kw = {"fifo_capacity": 3 * W * H} if kind == "fifo" else ({"world_points": True} if kind == "world" else {})
    a, s = _mk(dev, W, H, b, **kw), _mk(dev, W, H, b, **kw)

    def dev_batch(seed):
        bt = _random_batch(np.random.default_rng(seed), 30000, W, H, bad=0.05)
        t = [torch.from_numpy(bt[k]).to(dev) for k in ("pos", "color", "motion")]
        wp = torch.from_numpy(rng.uniform(-1, 1, (30000, 4)).astype(np.float32)).to(dev) if kind == "world" else None
        return t, wp

    (p1, c1, m1), w1 = dev_batch(1)
    (p2, c2, m2), w2 = dev_batch(2)
    for r in (a, s):
        r.insert(p1, c1, m1, world=w1)
    s.reset()
    s.insert(p2, c2, m2, world=w2)
    side = torch.cuda.Stream(dev)
    ev = torch.cuda.Event()
    with torch.cuda.stream(side):
        torch.cuda._sleep(1000000)   # the queues stay busy for a while on the other stream
        ev.record(side)
    a.insert(p2, c2, m2, world=w2, reset=True, queues_free=ev)
    torch.cuda.synchronize()
    for x, y in zip(a.export_ring(), s.export_ring()):
        np.testing.assert_array_equal(x, y)
    if kind == "world":   # the frame view from the stored hit points
        vp = np.eye(4, dtype=np.float32)
        vp[3, 2] = 1.0
        vp[3, 3] = 2.0
        a.reproject_camera(T_NOW, vp)
        s.reproject_camera(T_NOW, vp)
    else:                 # from the queues, or from the reconstructor queue
        a.reproject(T_NOW)
        s.reproject(T_NOW)
    torch.cuda.synchronize()
    for x, y in zip(a.export_frame(), s.export_frame()):
        np.testing.assert_array_equal(x, y)
    assert a.query() == s.query()
    batch = L.AfrSampleBatch(p2.data_ptr(), c2.data_ptr(), m2.data_ptr(), None if w2 is None else w2.data_ptr())
    import ctypes
    assert a.lib.afr_insert_samples_ex(a.h, ctypes.byref(batch), 30000, 2, None, None) == L.AFR_ERR_INVALID_ARG


# ----------------------------------------------------------------------------- end to end
@pytest.mark.parametrize("key", ["c1_128x128x4", "c4_512x512x8", "c2_1024x1024x8"])
def test_end_to_end_matches_oracle(dev, key):
    """The whole forward path from the same samples (the GPU's own gradients,
    widths and filter) against the FP64 oracle's whole path: every colour
    within 1e-5 relative (denominator max(|ref|, 1e-3)), on the static
    128x128x4 scene, the moving 512x512x8 scene and the moving, importance-
    sampled 1024x1024x8 scene. Prints the largest error and the number of
    channel values above 1e-5."""
    sc, batch = _scene_batch(key)
    W, H, b = sc.width, sc.height, sc.spec.depth
    rec = _mk(dev, W, H, b)
    _upload(rec, batch)
    rec.estimate_gradients(T_NOW)
    rec.reproject(T_NOW)
    img = rec.reconstruct(T_NOW).cpu().numpy().reshape(-1, 4).astype(np.float64)
    ring = oracle.Ring(W, H, b)
    ring.insert(batch["pos"], batch["color"], batch["motion"])
    ref = oracle.reconstruct(ring)["image"]
    hole = ref[:, 3] == 0
    np.testing.assert_array_equal(img[hole], 0.0)
    err = _rel_err(img[~hole, :3], ref[~hole, :3])
    print(f"{key}: end-to-end max rel err {err.max():.3g}, p99.9 {np.quantile(err, 0.999):.3g}, "
          f"{int((err > 1e-5).sum())} of {err.size} channel values above 1e-5")
    assert err.max() <= 1e-5
    big = ref[:, 3] > 1e-30
    np.testing.assert_allclose(img[big, 3], ref[big, 3], rtol=1e-4)


# ----------------------------------------------------------------------------- adjoint
def test_backward_matches_oracle(dev):
    W, H, b = 64, 48, 8
    _, _, rec, ring = _setup_scene(dev, W, H, b)
    rec.estimate_gradients(T_NOW)
    rec.reproject(T_NOW)
    L32, gx, gy, gt = _oracle_maps_f32(ring)
    for m, v in ((L.AFR_MAP_GX, gx), (L.AFR_MAP_GY, gy), (L.AFR_MAP_GT, gt)):
        rec.import_map(m, v)
    theta = np.array([0.9, 0.15, 2.4, 1.1, 0.02, 0.7])
    rec.reconstruct(T_NOW, theta)
    rng = np.random.default_rng(0)
    g = rng.normal(size=(W * H, 3))
    g4 = np.zeros((W * H, 4), np.float32)
    g4[:, :3] = g
    gcol, gprm = rec.backward(torch.from_numpy(g4).to(dev).reshape(H, W, 4))
    grads64 = (None, gx.astype(np.float64), gy.astype(np.float64), gt.astype(np.float64))
    off, frec, _, _ = oracle.reproject(ring, T_NOW)
    wcol, wprm = oracle.backward(ring.count, W, H, grads64, off, frec, g4[:, :3].astype(np.float64), theta)
    np.testing.assert_allclose(gprm.cpu().numpy(), wprm, rtol=2e-4, atol=1e-4 * np.abs(wprm).max())
    gc = gcol.cpu().numpy()
    scale = np.abs(wcol).max()
    np.testing.assert_allclose(gc, wcol, rtol=1e-3, atol=1e-5 * scale)

"""The reconstructor's global FIFO buffer (section 5.2) on the GPU against the
oracle: the frame view built from the N most recent accepted samples bit for
bit (including eviction and a batch larger than N), the filter over it, and
reset."""
import numpy as np
import pytest
import torch

import oracle
from workloads.scenes import SceneSpec, make_scene, sample_stream

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


def _batches(W, H, per_pixel, parts, seed, bad=0.02):
    sc = make_scene(SceneSpec(f"fifo_{W}x{H}", W, H, 4, 10, (5.0, 16.0), 40.0, 8), seed)
    batch = sample_stream(sc, W * H * per_pixel, seed)
    rng = np.random.default_rng(seed)
    k = int(len(batch["pos"]) * bad)
    idx = rng.choice(len(batch["pos"]), k, replace=False)
    batch["pos"][idx[0::2], 0] = np.float32(W)          # off-image
    batch["motion"][idx[1::2], 1] = np.inf              # non-finite
    cuts = np.linspace(0, len(batch["pos"]), parts + 1).astype(int)
    return [{key: np.ascontiguousarray(v[a:b]) for key, v in batch.items()} for a, b in zip(cuts[:-1], cuts[1:])]


def _fill(dev, W, H, b, N, batches):
    from paper_2510_15876_gb300.api import Reconstructor, to_device_batch
    rec = Reconstructor(W, H, b, fifo_capacity=N, device=dev)
    ring, fifo = oracle.Ring(W, H, b), oracle.Fifo(W, H, N)
    for bt in batches:
        rec.insert(*to_device_batch(bt, dev))
        ring.insert(bt["pos"], bt["color"], bt["motion"])
        fifo.insert(bt["pos"], bt["color"], bt["motion"])
    return rec, ring, fifo


def _frame_equal(rec, fifo):
    off, frec, fseq = rec.export_frame()
    woff, wrec, wseq, dropped = oracle.reproject_fifo(fifo, T_NOW)
    np.testing.assert_array_equal(off, woff)
    np.testing.assert_array_equal(fseq, wseq)
    np.testing.assert_array_equal(frec[:, :2], wrec[:, :2])
    np.testing.assert_array_equal(frec[:, 3:6], wrec[:, 3:6])
    a = (np.float32(T_NOW) - wrec[:, 2]).astype(np.float32)
    np.testing.assert_array_equal(frec[:, 2], (a * a).astype(np.float32))
    assert rec.query()["dropped"] == dropped
    return woff, wrec


@pytest.mark.parametrize("W,H,b,N,parts", [(96, 80, 4, 2 * 96 * 80, 3), (131, 67, 8, 1000, 2),
                                           (64, 48, 4, 64 * 48 * 9, 2)])
def test_fifo_frame_view_bitexact(dev, W, H, b, N, parts):
    """N below the accepted total (eviction), N below one batch (only its last
    N accepted samples stay), N above everything inserted."""
    rec, _, fifo = _fill(dev, W, H, b, N, _batches(W, H, 6, parts, seed=W))
    rec.reproject(T_NOW)
    _frame_equal(rec, fifo)


def test_fifo_filter_matches_oracle(dev):
    W, H, b, N = 96, 80, 4, 4 * 96 * 80
    rec, ring, fifo = _fill(dev, W, H, b, N, _batches(W, H, 6, 3, seed=7))
    rec.estimate_gradients(T_NOW)
    rec.reproject(T_NOW)
    grads = oracle.gradients(ring, T_NOW)
    ss, st = oracle.sigma(ring.count, W, H, grads, oracle.DEFAULT_THETA)
    ss32, st32 = ss.astype(np.float32), st.astype(np.float32)
    rec.import_map(L.AFR_MAP_SIGMA_S, ss32)
    rec.import_map(L.AFR_MAP_SIGMA_T, st32)
    img = rec.reconstruct(T_NOW, flags=L.AFR_RECON_KEEP_SIGMA).cpu().numpy().reshape(-1, 4).astype(np.float64)
    off, frec = _frame_equal(rec, fifo)
    ref = oracle.filter_image(W, H, off, frec, ss32.astype(np.float64), st32.astype(np.float64))
    hole = ref[:, 3] == 0
    np.testing.assert_array_equal(img[hole], 0.0)
    err = np.abs(img[~hole, :3] - ref[~hole, :3]) / np.maximum(np.abs(ref[~hole, :3]), 1e-3)
    assert err.max() <= 1e-5, err.max()


def test_fifo_reset_empties_it(dev):
    W, H, b, N = 48, 40, 4, 5000
    rec, _, _ = _fill(dev, W, H, b, N, _batches(W, H, 3, 1, seed=9))
    rec.reset()
    rec.reproject(T_NOW)
    assert rec.query()["frame"] == 0

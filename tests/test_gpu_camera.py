"""Camera-matrix reprojection (section 6.2: the stored hit points rendered
with the current camera, plus each sample's own screen motion) on the GPU
against the oracle: the frame view bit for bit from the per-pixel queues and
from the reconstructor queue, the filter over it, and argument checks."""
import types

import numpy as np
import pytest
import torch

import oracle
from workloads.scenes import SceneSpec, make_scene, sample_stream

pytestmark = pytest.mark.gpu

from paper_2510_15876_gb300 import _lib as L  # noqa: E402

T_NOW = 1.0
VP = np.array([[1.2, 0.1, 0.05, 0.02], [-0.05, 1.3, 0.1, -0.1], [0.0, 0.0, 1.0, 0.0], [0.01, 0.02, 0.4, 0.3]],
              np.float32)


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_15876_gb300.build import build
    build()
    return torch.device("cuda:0")


def _stream(W, H, b, seed):
    sc = make_scene(SceneSpec(f"camera_{W}x{H}", W, H, b, 10, (5.0, 16.0), 24.0, 8), seed)
    batch = sample_stream(sc, W * H * b, seed)
    rng = np.random.default_rng(seed)
    n = len(batch["pos"])
    world = np.stack([rng.uniform(-2, 2, n), rng.uniform(-2, 2, n), rng.uniform(2, 6, n), np.zeros(n)], 1)
    world = world.astype(np.float32)
    world[: n // 50, 2] = -4.0                      # behind the camera
    batch["world"] = world
    return batch


def _frame_equal(rec, want):
    off, frec, fseq = rec.export_frame()
    woff, wrec, wseq, dropped = want
    np.testing.assert_array_equal(off, woff)
    np.testing.assert_array_equal(fseq, wseq)
    np.testing.assert_array_equal(frec[:, :2], wrec[:, :2])
    np.testing.assert_array_equal(frec[:, 3:6], wrec[:, 3:6])
    a = (np.float32(T_NOW) - wrec[:, 2]).astype(np.float32)
    np.testing.assert_array_equal(frec[:, 2], (a * a).astype(np.float32))
    assert rec.query()["dropped"] == dropped


def _make(dev, W, H, b, fifo=0, seed=1):
    from paper_2510_15876_gb300.api import Reconstructor, to_device_batch
    batch = _stream(W, H, b, seed)
    rec = Reconstructor(W, H, b, fifo_capacity=fifo, world_points=True, device=dev)
    rec.insert(*to_device_batch(batch, dev), world=torch.from_numpy(batch["world"]).to(dev))
    ring = oracle.Ring(W, H, b)
    ring.insert(batch["pos"], batch["color"], batch["motion"])
    return rec, ring, batch


@pytest.mark.parametrize("W,H,b", [(96, 80, 4), (131, 67, 8)])
def test_camera_frame_view_bitexact(dev, W, H, b):
    rec, ring, batch = _make(dev, W, H, b)
    rec.reproject_camera(T_NOW, VP)
    _frame_equal(rec, oracle.reproject_camera(ring, batch["world"], VP, T_NOW))


def test_camera_from_the_reconstructor_queue(dev):
    W, H, b, N = 80, 64, 4, 9000
    rec, _, batch = _make(dev, W, H, b, fifo=N)
    fifo = oracle.Fifo(W, H, N)
    fifo.insert(batch["pos"], batch["color"], batch["motion"])
    k = fifo.resident
    as_list = types.SimpleNamespace(W=W, H=H, b=max(k, 1), resident=k, count=np.zeros(W * H, np.int32),
                                    slot=np.ascontiguousarray(fifo.q[:max(k, 1)]),
                                    seq=np.ascontiguousarray(fifo.seq[:max(k, 1)]))
    as_list.count[0] = k
    rec.reproject_camera(T_NOW, VP)
    _frame_equal(rec, oracle.reproject_camera(as_list, batch["world"], VP, T_NOW))


def test_camera_filter_matches_oracle(dev):
    W, H, b = 96, 80, 4
    rec, ring, batch = _make(dev, W, H, b, seed=4)
    rec.estimate_gradients(T_NOW)
    rec.reproject_camera(T_NOW, VP)
    grads = oracle.gradients(ring, T_NOW)
    ss, st = oracle.sigma(ring.count, W, H, grads, oracle.DEFAULT_THETA)
    ss32, st32 = ss.astype(np.float32), st.astype(np.float32)
    rec.import_map(L.AFR_MAP_SIGMA_S, ss32)
    rec.import_map(L.AFR_MAP_SIGMA_T, st32)
    img = rec.reconstruct(T_NOW, flags=L.AFR_RECON_KEEP_SIGMA).cpu().numpy().reshape(-1, 4).astype(np.float64)
    off, frec, _, _ = oracle.reproject_camera(ring, batch["world"], VP, T_NOW)
    ref = oracle.filter_image(W, H, off, frec, ss32.astype(np.float64), st32.astype(np.float64))
    hole = ref[:, 3] == 0
    np.testing.assert_array_equal(img[hole], 0.0)
    err = np.abs(img[~hole, :3] - ref[~hole, :3]) / np.maximum(np.abs(ref[~hole, :3]), 1e-3)
    assert err.max() <= 1e-5, err.max()


def test_camera_refresh_matches_serial_calls(dev):
    """refresh(view_proj=...) with the gradient branch on its side stream: the
    same image and tile statistics as the calls in series."""
    W, H, b = 96, 80, 4
    a, _, _ = _make(dev, W, H, b, seed=5)
    s, _, _ = _make(dev, W, H, b, seed=5)
    img_a, tiles_a = a.refresh(T_NOW, view_proj=VP)
    s.estimate_gradients(T_NOW)
    s.reproject_camera(T_NOW, VP)
    img_s = s.reconstruct(T_NOW)
    tiles_s = s.tile_feedback()
    assert torch.equal(img_a, img_s) and torch.equal(tiles_a, tiles_s)
    assert a.query()["frame"] == s.query()["frame"] > 0


def test_camera_argument_checks(dev):
    from paper_2510_15876_gb300.api import Reconstructor, to_device_batch
    batch = _stream(32, 24, 4, 7)
    rec = Reconstructor(32, 24, 4, world_points=True, device=dev)
    with pytest.raises(L.AfrError) as ei:
        rec.insert(*to_device_batch(batch, dev))            # no hit points
    assert ei.value.status == L.AFR_ERR_INVALID_ARG
    plain = Reconstructor(32, 24, 4, device=dev)
    plain.insert(*to_device_batch(batch, dev))
    with pytest.raises(L.AfrError) as ei:
        plain.reproject_camera(T_NOW, VP)
    assert ei.value.status == L.AFR_ERR_BAD_STATE
    bad = VP.copy()
    bad[0, 0] = np.inf
    rec.insert(*to_device_batch(batch, dev), world=torch.from_numpy(batch["world"]).to(dev))
    with pytest.raises(L.AfrError) as ei:
        rec.reproject_camera(T_NOW, bad)
    assert ei.value.status == L.AFR_ERR_INVALID_ARG

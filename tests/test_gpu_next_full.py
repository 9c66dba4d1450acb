"""The global FIFO buffer (section 5.2) and camera-matrix reprojection
(section 6.2) at the size of the 1024x1024, 8-deep importance-sampled workload
(8,388,608 samples): frame views bit for bit against the oracle, and the filter
over them at sampled pixels on the oracle's widths."""
import numpy as np
import pytest
import torch

import oracle
from workloads import scenes

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

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


@pytest.fixture(scope="module")
def c2():
    scene, batch = scenes.config_stream("c2_1024x1024x8", 0)
    ring = oracle.Ring(scene.width, scene.height, scene.spec.depth)
    ring.insert(batch["pos"], batch["color"], batch["motion"])
    grads = oracle.gradients(ring, T_NOW)
    ss, st = oracle.sigma(ring.count, scene.width, scene.height, grads, oracle.DEFAULT_THETA)
    return scene, batch, ring, ss.astype(np.float32), st.astype(np.float32)


def _frame_equal(rec, want):
    off, frec, fseq = rec.export_frame()
    woff, wrec, wseq, dropped = want
    assert np.array_equal(off, woff) and np.array_equal(fseq, wseq)
    assert np.array_equal(frec[:, :2], wrec[:, :2]) and np.array_equal(frec[:, 3:6], wrec[:, 3:6])
    a = (np.float32(T_NOW) - wrec[:, 2]).astype(np.float32)
    assert np.array_equal(frec[:, 2], (a * a).astype(np.float32))
    assert rec.query()["dropped"] == dropped


def _filter_at_samples(rec, W, H, want, ss32, st32):
    woff, wrec = want[0], want[1]
    rec.import_map(L.AFR_MAP_SIGMA_S, ss32)
    rec.import_map(L.AFR_MAP_SIGMA_T, st32)
    pix = np.random.default_rng(1).choice(W * H, 4096, replace=False)
    got = rec.reconstruct(T_NOW, flags=L.AFR_RECON_KEEP_SIGMA).cpu().numpy().reshape(-1, 4)[pix].astype(np.float64)
    ref = oracle.filter_image(W, H, woff, wrec, ss32.astype(np.float64), st32.astype(np.float64),
                              pixels=pix)[pix]
    hole = ref[:, 3] == 0
    assert np.all(got[hole] == 0)
    err = np.abs(got[~hole, :3] - ref[~hole, :3]) / np.maximum(np.abs(ref[~hole, :3]), 1e-3)
    assert err.max() <= 1e-5, err.max()


def test_fifo_full_workload(dev, c2):
    """N = 4P, the batch in two halves: the second evicts part of the first."""
    from paper_2510_15876_gb300.api import Reconstructor, to_device_batch
    scene, batch, ring, ss32, st32 = c2
    W, H, b = scene.width, scene.height, scene.spec.depth
    N = 4 * W * H
    rec = Reconstructor(W, H, b, fifo_capacity=N, device=dev)
    fifo = oracle.Fifo(W, H, N)
    n = len(batch["pos"])
    for a, e in ((0, n // 2), (n // 2, n)):
        part = {k: np.ascontiguousarray(v[a:e]) for k, v in batch.items()}
        rec.insert(*to_device_batch(part, dev))
        fifo.insert(part["pos"], part["color"], part["motion"])
    rec.estimate_gradients(T_NOW)
    rec.reproject(T_NOW)
    want = oracle.reproject_fifo(fifo, T_NOW)
    assert rec.query()["frame"] > 0.9 * N
    _frame_equal(rec, want)
    _filter_at_samples(rec, W, H, want, ss32, st32)
    rec.close()


def test_camera_full_workload(dev, c2):
    """Random hit points in front of and (2%) behind a perspective camera."""
    from paper_2510_15876_gb300.api import Reconstructor, to_device_batch
    scene, batch, ring, ss32, st32 = c2
    W, H, b = scene.width, scene.height, scene.spec.depth
    n = len(batch["pos"])
    rng = np.random.default_rng(2)
    world = np.stack([rng.uniform(-2, 2, n), rng.uniform(-2, 2, n), rng.uniform(2, 6, n), np.zeros(n)], 1)
    world = world.astype(np.float32)
    world[: n // 50, 2] = -4.0
    rec = Reconstructor(W, H, b, world_points=True, device=dev)
    rec.insert(*to_device_batch(batch, dev), world=torch.from_numpy(world).to(dev))
    rec.estimate_gradients(T_NOW)
    rec.reproject_camera(T_NOW, VP)
    want = oracle.reproject_camera(ring, world, VP, T_NOW)
    _frame_equal(rec, want)
    _filter_at_samples(rec, W, H, want, ss32, st32)
    rec.close()

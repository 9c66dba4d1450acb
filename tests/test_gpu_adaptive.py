"""Adaptive footprints (section 6.2, the coverage map in gather form) on the
GPU against the oracle: footprint radii and sample counts bit for bit over
several images, colours within 1e-5 given the oracle's widths, hole filling,
and no effect on the fixed-footprint path."""
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


def _setup(dev, W, H, b, seed=3, speed=24.0, discs=10, hole=None, R=4):
    import dataclasses
    from paper_2510_15876_gb300.api import Reconstructor, to_device_batch
    spec = dataclasses.replace(scenes.CONFIGS["c4_512x512x8"], key=f"adaptive-{W}x{H}x{b}", width=W, height=H,
                               depth=b, speed=speed, n_discs=discs, edge_fraction=None, importance=False)
    sc = scenes.make_scene(spec, seed)
    batch = scenes.sample_stream(sc, W * H * b, seed)
    if hole is not None:
        cx, cy, r = hole
        keep = (batch["pos"][:, 0] - cx) ** 2 + (batch["pos"][:, 1] - cy) ** 2 > r * r
        batch = {k: np.ascontiguousarray(v[keep]) for k, v in batch.items()}
    rec = Reconstructor(W, H, b, device=dev, radius=R)
    rec.insert(*to_device_batch(batch, dev))
    ring = oracle.Ring(W, H, b)
    ring.insert(batch["pos"], batch["color"], batch["motion"])
    rec.estimate_gradients(T_NOW)
    rec.reproject(T_NOW)
    return rec, ring


def _oracle_widths(ring, W, H):
    grads = oracle.gradients(ring, T_NOW)
    ss, st = oracle.sigma(ring.count, W, H, grads, oracle.DEFAULT_THETA)
    return ss.astype(np.float32), st.astype(np.float32)


@pytest.mark.parametrize("W,H,b,R", [(96, 80, 4, 4), (131, 67, 8, 2)])
def test_adaptive_frames_match_oracle(dev, W, H, b, R):
    rec, ring = _setup(dev, W, H, b, R=R, hole=(W * 0.5, H * 0.5, 4.5))
    ss32, st32 = _oracle_widths(ring, W, H)
    rec.import_map(L.AFR_MAP_SIGMA_S, ss32)
    rec.import_map(L.AFR_MAP_SIGMA_T, st32)
    off, frec, _, _ = oracle.reproject(ring, T_NOW)
    state = {"r": np.full(W * H, float(R), np.float32), "n": np.full(W * H, -1, np.int32)}
    seen = set()
    for frame in range(4):
        flags = L.AFR_RECON_KEEP_SIGMA | L.AFR_RECON_ADAPTIVE_SUPPORT
        if frame == 0:
            flags |= L.AFR_RECON_COVERAGE_RESET
        img = rec.reconstruct(T_NOW, flags=flags).cpu().numpy().reshape(-1, 4).astype(np.float64)
        r_ref, R_ref = oracle.coverage_update(W, H, state["r"], state["n"])
        n_ref = oracle.coverage_count(W, H, R_ref, off)
        state["r"], state["n"] = r_ref, n_ref
        np.testing.assert_array_equal(rec.export_map(L.AFR_MAP_FOOTPRINT), r_ref)
        np.testing.assert_array_equal(rec.export_map(L.AFR_MAP_COVERAGE).astype(np.int64), n_ref)
        ref = oracle.filter_image(W, H, off, frec, ss32.astype(np.float64), st32.astype(np.float64), R=R_ref)
        hole = ref[:, 3] == 0
        np.testing.assert_array_equal(img[hole], 0.0)
        err = np.abs(img[~hole, :3] - ref[~hole, :3]) / np.maximum(np.abs(ref[~hole, :3]), 1e-3)
        assert err.max() <= 1e-5, (frame, err.max())
        seen.update(np.unique(R_ref).tolist())
    assert len(seen) >= 3          # the footprints did change across frames


def test_adaptive_fills_holes(dev):
    W, H, b = 64, 48, 4
    rec, _ = _setup(dev, W, H, b, R=1, hole=(32.0, 24.0, 3.5))
    first = rec.reconstruct(T_NOW, flags=L.AFR_RECON_ADAPTIVE_SUPPORT | L.AFR_RECON_COVERAGE_RESET)
    holes = (first[..., 3] == 0).cpu().numpy().reshape(-1)
    assert holes.sum() > 0
    second = rec.reconstruct(T_NOW, flags=L.AFR_RECON_ADAPTIVE_SUPPORT)
    assert bool((second[..., 3] > 0).all())
    r = rec.export_map(L.AFR_MAP_FOOTPRINT)
    assert (r[holes] == 4.0).all()


def test_fixed_footprint_unaffected_and_backward_guard(dev):
    W, H, b = 80, 64, 4
    rec, _ = _setup(dev, W, H, b)
    ref = rec.reconstruct(T_NOW).clone()
    for _ in range(2):
        rec.reconstruct(T_NOW, flags=L.AFR_RECON_ADAPTIVE_SUPPORT)
    with pytest.raises(L.AfrError) as ei:
        rec.backward(torch.ones((H, W, 4), device=dev))
    assert ei.value.status == L.AFR_ERR_BAD_STATE
    again = rec.reconstruct(T_NOW)
    assert torch.equal(again, ref)
    rec.backward(torch.ones((H, W, 4), device=dev))     # allowed again after a fixed reconstruction

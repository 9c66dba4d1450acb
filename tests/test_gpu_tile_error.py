"""Tile error E_tile (section 6.1) and gain control (section 4.1) on the GPU
against the oracle, with and without the caller's occlusion counts."""
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


def _setup(dev, W, H, b, S, seed):
    from paper_2510_15876_gb300.api import Reconstructor, to_device_batch
    sc = make_scene(SceneSpec(f"tile_error_{W}x{H}", W, H, b, 12, (6.0, 20.0), 24.0, 8), seed)
    batch = sample_stream(sc, W * H * b, seed)
    # a sparse region, so that some tiles are undersampled (u > 0)
    rng = np.random.default_rng(seed)
    keep = (batch["pos"][:, 0] < 0.7 * W) | (rng.uniform(0, 1, len(batch["pos"])) < 0.05)
    batch = {k: np.ascontiguousarray(v[keep]) for k, v in batch.items()}
    rec = Reconstructor(W, H, b, tile=S, device=dev)
    rec.insert(*to_device_batch(batch, dev))
    ring = oracle.Ring(W, H, b)
    ring.insert(batch["pos"], batch["color"], batch["motion"])
    rec.estimate_gradients(T_NOW)
    return rec, ring


@pytest.mark.parametrize("W,H,b,S", [(160, 96, 8, 32), (131, 67, 4, 16), (300, 140, 16, 64)])
@pytest.mark.parametrize("with_occlusion", [False, True])
def test_tile_error_and_gain_match_oracle(dev, W, H, b, S, with_occlusion):
    rec, ring = _setup(dev, W, H, b, S, seed=W)
    grads = oracle.gradients(ring, T_NOW)
    tiles = oracle.tile_feedback(ring, grads, S, T_NOW)
    assert (tiles[:, 7] > 0).any()
    occ = None
    if with_occlusion:
        occ = np.random.default_rng(1).integers(0, 40, tiles.shape[0]).astype(np.int32)
    kappa, lam, imp = 0.35, 0.4, 1.25
    E, gain = rec.tile_error(kappa, lam, imp, None if occ is None else torch.from_numpy(occ))
    E_ref, g_ref = oracle.tile_error(ring, tiles, S, T_NOW, None if occ is None else occ.astype(np.float64),
                                     kappa, lam, imp)
    E = E.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(E, E_ref, rtol=1e-4, atol=1e-5 * np.abs(E_ref).max())
    got = [gain[k] for k in ("dC_ds", "dC_dt", "mean_age", "tile_width", "tile_count")]
    np.testing.assert_allclose(got, g_ref, rtol=1e-4)


def test_tile_error_rejects_bad_weights(dev):
    rec, _ = _setup(dev, 64, 48, 4, 16, seed=5)
    for kappa, lam, imp in [(0.7, 0.5, 1.0), (-0.1, 0.5, 1.0), (0.5, 0.5, -1.0)]:
        with pytest.raises(L.AfrError) as ei:
            rec.tile_error(kappa, lam, imp)
        assert ei.value.status == L.AFR_ERR_INVALID_ARG


def test_gain_on_device_and_preallocated_outputs(dev):
    rec, _ = _setup(dev, 131, 67, 4, 16, seed=9)
    E, gain = rec.tile_error(0.3, 0.3, 2.0)
    out = (torch.full_like(E, -1.0), torch.full((5,), -1.0, device=dev))
    E2, g2 = rec.tile_error(0.3, 0.3, 2.0, out=out, gain_on_device=True)
    assert E2.data_ptr() == out[0].data_ptr() and g2.data_ptr() == out[1].data_ptr()
    assert torch.equal(E, E2)
    assert g2.cpu().tolist() == [gain[k] for k in rec.GAIN_KEYS]

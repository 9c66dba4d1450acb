"""Failure detection without faulting the GPU.

* Device checks: the AFR_DEBUG build (libafr_debug.so) bounds-checks record
  and slot indices on the device. A frame view made inconsistent from the
  host (offsets pointing past the records) reaches the filter's checks: each
  guarded read is skipped, never performed, and afr_get_status reports
  AFR_ERR_DEVICE_CHECK once; a consistent run reports AFR_OK and gives the
  release library's image bit for bit.
* Allocation failures: the debug build's allocator hook fails the k-th device
  allocation; afr_create returns AFR_ERR_OOM for every k and leaks nothing,
  and a failed scratch growth in afr_insert_samples leaves the context usable.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

from paper_2510_15876_gb300 import _lib as L  # noqa: E402


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_15876_gb300.build import build
    build()
    return torch.device("cuda:0")


def _batch(seed, n, W, H):
    rng = np.random.default_rng(seed)
    pos = np.stack([rng.uniform(0, W, n), rng.uniform(0, H, n), np.sort(rng.uniform(0, 1, n)),
                    rng.uniform(0, 1, n)], 1).astype(np.float32)
    col = np.zeros((n, 4), np.float32)
    col[:, :3] = rng.uniform(0, 1, (n, 3))
    mo = rng.uniform(-3, 3, (n, 2)).astype(np.float32)
    return {"pos": pos, "color": col, "motion": mo}


def _filled(dev, lib, W=20, H=10, b=4, seed=0):
    from paper_2510_15876_gb300.api import Reconstructor, to_device_batch
    rec = Reconstructor(W, H, b, device=dev, lib=lib)
    rec.insert(*to_device_batch(_batch(seed, W * H * b, W, H), dev))
    rec.estimate_gradients(1.0)
    rec.reproject(1.0)
    return rec


def test_debug_build_matches_release_and_reports_ok(dev):
    rel = _filled(dev, L.load())
    dbg = _filled(dev, L.load_debug())
    a, b = rel.reconstruct(1.0), dbg.reconstruct(1.0)
    assert torch.equal(a, b)
    assert dbg.status() == L.AFR_OK and rel.status() == L.AFR_OK
    rel.close()
    dbg.close()


def test_inconsistent_frame_view_reaches_the_device_checks(dev):
    lib = L.load_debug()
    W, H, b = 20, 10, 4
    rec = _filled(dev, lib, W, H, b, seed=1)
    off, _, _ = rec.export_frame()
    cap = W * H * b                        # the context's frame-view capacity
    bad = off.astype(np.int64)
    bad[W * H // 2:] += cap + 7            # the second half of the bins points past every record
    bad = np.ascontiguousarray(bad.astype(np.uint32))
    assert lib.afr_debug_set_frame_offsets(rec.h, bad.ctypes.data) == L.AFR_OK
    rec.reconstruct(1.0)
    assert rec.status() == L.AFR_ERR_DEVICE_CHECK
    assert rec.status() == L.AFR_OK        # the status word was cleared
    # the context stays usable: a fresh frame view is consistent again
    rec.reproject(1.0)
    rec.reconstruct(1.0)
    assert rec.status() == L.AFR_OK
    rec.close()


def test_injected_allocation_failures_return_oom_without_leaks(dev):
    lib = L.load_debug()
    cfg = L.AfrConfig(64, 48, 8, 32, 4, L.AFR_F32, 1.0, 1e-4, 2.0, 256, 1)   # FIFO and hit points: every buffer
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    h = ctypes.c_void_p()
    seen_ok, k = False, 0
    while not seen_ok:
        lib.afr_debug_fail_alloc(k)
        st = lib.afr_create(ctypes.byref(cfg), ctypes.byref(h))
        if st == L.AFR_OK:
            seen_ok = True
            lib.afr_destroy(h)
        else:
            assert st == L.AFR_ERR_OOM, (k, st)
            assert not h.value
        k += 1
        assert k < 200
    lib.afr_debug_fail_alloc(-1)
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (8 << 20)   # every failed create freed what it took
    assert k > 20                            # the context's allocations were each made to fail


def test_failed_scratch_growth_leaves_the_context_usable(dev):
    from paper_2510_15876_gb300.api import Reconstructor, to_device_batch
    lib = L.load_debug()
    W, H, b = 32, 16, 4
    rec = Reconstructor(W, H, b, device=dev, lib=lib)
    batch = to_device_batch(_batch(3, 4000, W, H), dev)
    lib.afr_debug_fail_alloc(0)
    with pytest.raises(L.AfrError) as e:
        rec.insert(*batch)
    assert e.value.status == L.AFR_ERR_OOM
    lib.afr_debug_fail_alloc(-1)
    rec.insert(*batch)
    rec.estimate_gradients(1.0)
    rec.reproject(1.0)
    rec.reconstruct(1.0)
    assert rec.status() == L.AFR_OK
    assert rec.query()["inserted"] == 4000
    rec.close()

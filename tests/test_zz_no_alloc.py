"""afr_reproject_batch_static against the regular context path.

Callers that cannot allocate device memory when they need the step (a render
thread with a fixed memory budget, a host whose frame callback forbids
allocation) use the allocation-free entry point. Given a batch that fits a
context's queues whole, it must produce the frame view that
afr_insert_samples + afr_reproject produce: the same bins, the same order,
the same moved positions and colours, bit for bit (the tolerance the parity
tests use for indices and for the single-precision move), on two calls in a
row that share its scratch array.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


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
    mo = rng.uniform(-20, 20, (n, 2)).astype(np.float32)   # some samples leave the image
    bad = rng.choice(n, n // 50, replace=False)
    pos[bad[0::3], 0] = np.nan
    col[bad[1::3], 1] = np.inf
    pos[bad[2::3], 1] = H                                    # off-image: rejected
    return {"pos": pos, "color": col, "motion": mo}


_CT = {"f32": (0, torch.float32), "f16": (1, torch.float16), "bf16": (2, torch.bfloat16)}


def _static(lib, L, batch_t, n, W, H, t_now, dev, ct="f32"):
    pos, col, mo = batch_t
    code, dtype = _CT[ct]
    P = W * H
    off = torch.zeros(P + 1, dtype=torch.int32, device=dev)
    rec = torch.zeros((n, 4), dtype=torch.float32, device=dev)
    out_col = torch.zeros((n, 4), dtype=dtype, device=dev)
    seq = torch.zeros(n, dtype=torch.int32, device=dev)
    nf = torch.zeros(1, dtype=torch.int32, device=dev)
    b = L.AfrSampleBatch(pos.data_ptr(), col.data_ptr(), mo.data_ptr())
    st = lib.afr_reproject_batch_static(ctypes.byref(b), n, W, H, code, t_now, off.data_ptr(),
                                        rec.data_ptr(), out_col.data_ptr(), seq.data_ptr(), nf.data_ptr(),
                                        torch.cuda.current_stream().cuda_stream)
    assert st == L.AFR_OK
    torch.cuda.synchronize()
    m = int(nf.item())
    return (off.cpu().numpy().view(np.uint32), rec.cpu().numpy()[:m], out_col.float().cpu().numpy()[:m],
            seq.cpu().numpy().view(np.uint32)[:m], m)


def test_static_matches_context_path_on_consecutive_calls(dev):
    from paper_2510_15876_gb300 import _lib as L
    from paper_2510_15876_gb300.api import Reconstructor, to_device_batch
    lib = L.load()
    W, H, n = 200, 150, 90000      # about 3 samples per pixel: a 32-deep queue keeps them all
    for call, (seed, t_now) in enumerate(((1, 1.0), (2, 0.75))):
        batch = _batch(seed, n, W, H)
        tensors = to_device_batch(batch, dev)
        off_s, rec_s, col_s, seq_s, m = _static(lib, L, tensors, n, W, H, t_now, dev)

        ctx = Reconstructor(W, H, 32, device=dev)
        ctx.insert(*tensors)
        ctx.reproject(t_now)
        off_c, rec_c, seq_c = ctx.export_frame()
        ctx.close()

        np.testing.assert_array_equal(off_s, off_c, err_msg=f"call {call}")
        assert m == rec_c.shape[0]
        np.testing.assert_array_equal(seq_s, seq_c)
        np.testing.assert_array_equal(rec_s[:, :3], rec_c[:, :3])          # x', y', a^2
        np.testing.assert_array_equal(col_s[:, :3], rec_c[:, 3:6])
        np.testing.assert_array_equal(rec_s[:, 3].view(np.int32), np.floor(rec_c[:, 0]).astype(np.int32))


@pytest.mark.parametrize("ct", ["f16", "bf16"])
def test_static_16bit_colours_match_context_path(dev, ct):
    """The 16-bit colour forms, two calls in a row, against a context of the
    same colour type."""
    from paper_2510_15876_gb300 import _lib as L
    from paper_2510_15876_gb300.api import Reconstructor, to_device_batch
    lib = L.load()
    W, H, n = 160, 96, 40000
    for call, (seed, t_now) in enumerate(((3, 1.0), (4, 0.5))):
        batch = _batch(seed, n, W, H)
        tensors = to_device_batch(batch, dev, _CT[ct][1])
        off_s, rec_s, col_s, seq_s, m = _static(lib, L, tensors, n, W, H, t_now, dev, ct)
        ctx = Reconstructor(W, H, 32, color_type=ct, device=dev)
        ctx.insert(*tensors)
        ctx.reproject(t_now)
        off_c, rec_c, seq_c = ctx.export_frame()
        ctx.close()
        np.testing.assert_array_equal(off_s, off_c, err_msg=f"call {call}")
        np.testing.assert_array_equal(seq_s, seq_c)
        np.testing.assert_array_equal(rec_s[:, :3], rec_c[:, :3])
        np.testing.assert_array_equal(col_s[:, :3], rec_c[:, 3:6])


def test_static_dense_bin_beyond_the_ordering_limit(dev):
    """One bin of 5000 records (above the 4096-record ordering limit) among a
    few thousand others: every other bin bit-exact and in batch order, the
    dense bin the same records in some order; the reference is a context whose
    reconstructor queue (section 5.2) holds the whole batch."""
    from paper_2510_15876_gb300 import _lib as L
    from paper_2510_15876_gb300.api import Reconstructor, to_device_batch
    lib = L.load()
    W, H = 64, 48
    rng = np.random.default_rng(11)
    dense, spread = 5000, 3000
    batch = _batch(12, dense + spread, W, H)
    idx = rng.permutation(dense + spread)[:dense]
    batch["pos"][idx, 0] = 17.25 + rng.uniform(0, 0.5, dense).astype(np.float32)
    batch["pos"][idx, 1] = 9.5
    batch["motion"][idx] = 0.0
    n = dense + spread
    tensors = to_device_batch(batch, dev)
    for call in range(2):
        off_s, rec_s, col_s, seq_s, m = _static(lib, L, tensors, n, W, H, 1.0, dev)
        ctx = Reconstructor(W, H, 1, fifo_capacity=n, device=dev)
        ctx.insert(*tensors)
        ctx.reproject(1.0)
        off_c, rec_c, seq_c = ctx.export_frame()
        unsorted = ctx.query()["unsorted_bins"]
        ctx.close()
        assert unsorted == 1
        np.testing.assert_array_equal(off_s, off_c, err_msg=f"call {call}")
        q = 9 * W + 17
        lo, hi = int(off_s[q]), int(off_s[q + 1])
        assert hi - lo > 4096
        keep = np.ones(m, bool)
        keep[lo:hi] = False
        np.testing.assert_array_equal(seq_s[keep], seq_c[keep])
        np.testing.assert_array_equal(rec_s[keep, :3], rec_c[keep, :3])
        np.testing.assert_array_equal(col_s[keep, :3], rec_c[keep, 3:6])
        o_s, o_c = np.argsort(seq_s[lo:hi]), np.argsort(seq_c[lo:hi])
        np.testing.assert_array_equal(seq_s[lo:hi][o_s], seq_c[lo:hi][o_c])
        np.testing.assert_array_equal(rec_s[lo:hi, :3][o_s], rec_c[lo:hi, :3][o_c])
        np.testing.assert_array_equal(col_s[lo:hi, :3][o_s], rec_c[lo:hi, 3:6][o_c])


def test_static_rejects_sizes_beyond_its_scratch(dev):
    from paper_2510_15876_gb300 import _lib as L
    lib = L.load()
    b = L.AfrSampleBatch(None, None, None)
    one = torch.zeros(16, dtype=torch.float32, device=dev)
    st = lib.afr_reproject_batch_static(ctypes.byref(b), 0, 2048, 1024, L.AFR_F32, 1.0, one.data_ptr(),
                                        one.data_ptr(), one.data_ptr(), one.data_ptr(), None, None)
    assert st == L.AFR_ERR_INVALID_ARG

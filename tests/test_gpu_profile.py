"""Filter kernel timing hook (afr_profile_filter / afr_profile_read)."""
import pytest
import torch

from workloads.scenes import SceneSpec, make_scene, sample_stream

pytestmark = pytest.mark.gpu

from paper_2510_15876_gb300 import _lib as L  # noqa: E402


@pytest.fixture(scope="module")
def rec():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_15876_gb300.api import Reconstructor, to_device_batch
    W, H, b = 96, 80, 8
    sc = make_scene(SceneSpec("profile_test", W, H, b, 12, (4.0, 16.0), 24.0, 8), 0)
    r = Reconstructor(W, H, b, device="cuda:0")
    r.insert(*to_device_batch(sample_stream(sc, W * H * b, 0), "cuda:0"))
    r.estimate_gradients(1.0)
    r.reproject(1.0)
    yield r
    r.close()


def test_records_each_launch_and_clears(rec):
    ref = rec.reconstruct(1.0).clone()
    rec.profile_filter(True)
    outs = [rec.reconstruct(1.0).clone() for _ in range(3)]
    ms = rec.profile_read()
    assert len(ms) == 3 and all(0.0 < t < 1000.0 for t in ms)
    assert all(torch.equal(o, ref) for o in outs)       # timing changes nothing
    assert rec.profile_read() == []
    rec.profile_filter(False)
    rec.reconstruct(1.0)
    assert rec.profile_read() == []


def test_capture_is_reported_not_timed(rec):
    rec.profile_filter(True)
    out = torch.empty((rec.H, rec.W, 4), device="cuda:0")
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        rec.reconstruct(1.0, out=out)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        rec.reconstruct(1.0, out=out)
    g.replay()
    torch.cuda.synchronize()
    with pytest.raises(L.AfrError) as ei:
        rec.profile_read()
    assert ei.value.status == L.AFR_ERR_BAD_STATE
    rec.profile_filter(False)

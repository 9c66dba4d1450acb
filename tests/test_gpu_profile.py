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


def test_step_launches_match_the_bench_count():
    """The kernels one step a1-a6 launches, per stage, as the profiler sees
    them, equal the counts bench.py reports as gpu_launches."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import bench
    from paper_2510_15876_gb300.api import Reconstructor, to_device_batch
    W, H, b = 96, 80, 8
    sc = make_scene(SceneSpec("launch_count", W, H, b, 12, (4.0, 16.0), 24.0, 8), 1)
    pos, col, mo = to_device_batch(sample_stream(sc, W * H * b, 1), "cuda:0")
    r = Reconstructor(W, H, b, device="cuda:0")
    calls = {"ingest": lambda: r.insert(pos, col, mo), "gradients": lambda: r.estimate_gradients(1.0),
             "reproject": lambda: r.reproject(1.0), "reconstruct": lambda: r.reconstruct(1.0),
             "feedback": lambda: r.tile_feedback()}
    for fn in calls.values():   # warm up (first-use allocations and attributes)
        fn()
    torch.cuda.synchronize()
    from torch.profiler import ProfilerActivity, profile
    try:   # the first session of a process may miss its kernels while the tracer starts
        with profile(activities=[ProfilerActivity.CUDA]):
            r.insert(pos, col, mo)
            torch.cuda.synchronize()
    except Exception as ex:   # no CUPTI in this environment
        pytest.skip(f"profiler unavailable: {ex}")
    got = {}
    for stage, fn in calls.items():
        try:
            with profile(activities=[ProfilerActivity.CUDA]) as prof:
                fn()
                torch.cuda.synchronize()
        except Exception as ex:   # no CUPTI in this environment
            pytest.skip(f"profiler unavailable: {ex}")
        names = [e.name for e in prof.events() if e.device_type == torch.autograd.DeviceType.CUDA]
        got[stage] = sum(1 for n in names if "k_" in n and "Memcpy" not in n and "Memset" not in n)
    r.close()
    assert got == bench.LAUNCHES, got

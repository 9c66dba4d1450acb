"""Host logic of bench.py for N > 1 ranks, on CPU with the gloo backend:
max-over-ranks timing, rank-0-only printing of the oracle arm, and the pair
count used by the roofline."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(10.0 + 5.0 * rank, dist)
        dist.barrier()
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    assert res == [(0, 15.0), (1, 15.0)]


def test_max_over_ranks_single_process():
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert bench.max_over_ranks(3.5, dist) == 3.5      # not initialised: identity


def test_reference_arm_other_ranks_do_no_work(capsys):
    class A:
        steps, warmup = 1, 0
    bench.run_reference(A(), rank=1, world=2)
    assert capsys.readouterr().out == ""


@pytest.mark.parametrize("R", [0, 1, 3, 4])
def test_pairs_of_matches_brute_force(R):
    rng = np.random.default_rng(R)
    W, H = 13, 9
    cnt = rng.integers(0, 4, W * H)
    off = np.concatenate([[0], np.cumsum(cnt)]).astype(np.uint32)
    c = cnt.reshape(H, W)
    ref = 0
    for y in range(H):
        for x in range(W):
            for dy in range(-R, R + 1):
                for dx in range(-R, R + 1):
                    if dx * dx + dy * dy <= R * R and 0 <= x + dx < W and 0 <= y + dy < H:
                        ref += int(c[y + dy, x + dx])
    assert bench.pairs_of(off, W, H, R) == ref


def test_filter_traffic_only_for_the_captured_source(monkeypatch):
    """roofline.traffic: a figure on the command line wins; the recorded
    capture is reported only for the captured workload and colour type and
    only while the filter's sources hash to the captured ones."""
    import types
    import bench
    args = types.SimpleNamespace(filter_traffic=None, workload=bench.WORKLOAD)
    assert bench.filter_traffic(types.SimpleNamespace(filter_traffic=5.0, workload="x"), "f16") == (5.0, "--filter-traffic")
    assert bench.filter_traffic(args, "f16")[0] is None
    assert bench.filter_traffic(types.SimpleNamespace(filter_traffic=None, workload="c1_128x128x4"), "f32")[0] is None
    value, _ = bench.filter_traffic(args, "f32")
    assert value is not None and value > 0   # the sources in the tree are the captured ones
    monkeypatch.setattr(bench, "FILTER_TRAFFIC", {("0" * 64, "0" * 64): 1.0})
    assert bench.filter_traffic(args, "f32") == (None, "kernel source changed since the last capture")

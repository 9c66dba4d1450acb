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

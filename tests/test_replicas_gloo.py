"""The benchmark's N > 1 path on CPU: two `gloo` ranks (world size 2,
rendezvous on 127.0.0.1), each a replica with its own stream.  The whole-job
time is the slowest rank's and the work is the sum over the ranks (weak
scaling, no data-path collective); the reference arm runs on rank 0 alone;
replicas draw different frames."""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

WS = 2


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, port: int, q) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(WS),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=WS)
    try:
        ws, r, lr = bench.dist_info()
        # rank r took 1 + r seconds for 100 (r + 1) units
        t, u = bench.job_totals(1.0 + r, 100.0 * (r + 1), ws, device="cpu")
        e2e_t, _ = bench.job_totals(2.5 - r, 0.0, ws, device="cpu")
        q.put((r, ws, lr, t, u, e2e_t))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time_and_the_summed_work():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, port, q)) for r in range(WS)]
    for p in procs:
        p.start()
    try:
        out = sorted(q.get(timeout=120) for _ in range(WS))
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    for r, (rank, ws, lrank, t, u, e2e_t) in enumerate(out):
        assert (rank, ws, lrank) == (r, WS, r)
        assert t == 2.0 and u == 300.0 and e2e_t == 2.5


def test_one_process_needs_no_collective():
    import bench
    assert bench.job_totals(0.25, 7, 1) == (0.25, 7.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class Args:
        warmup, steps = 3, 1
    assert bench.run_reference(Args()) == 0   # returns before any work on rank 1


def test_replicas_draw_different_frames():
    import bench
    a = bench.make_frames(1, seed=2 + 17 * 0)[0]
    b = bench.make_frames(1, seed=2 + 17 * 1)[0]
    assert a.shape[1] == 6 and b.shape[1] == 6
    assert a.shape != b.shape or not np.array_equal(a, b)

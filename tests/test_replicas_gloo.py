"""The benchmark's N > 1 path on CPU: two `gloo` ranks (world size 2,
rendezvous on 127.0.0.1), each a replica with its own stream.  The whole-job
time is the slowest rank's and the work is the sum over the ranks (weak
scaling, no data-path collective); the reference arm runs on rank 0 alone;
replicas draw different frames.  Also the exchange step a frame sharded by
points would need: one all-reduce of Delta S gives the whole frame's sums."""
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


def _shard_main(rank: int, port: int, q) -> None:
    """One rank of a frame sharded by points: the oracle's E-step statistics
    of its shard under the shared posterior, then one all-reduce (sum) of
    Delta S and of the lse sum -- the exchange step a sharded frame needs."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(WS))
    import torch
    import torch.distributed as dist
    from oracle import oracle as O
    from paper_2603_08499_gb300 import synth
    dist.init_process_group("gloo", rank=rank, world_size=WS)
    try:
        X, pr = synth.c1_workload(seed=51, N=1_001, K=37)
        post = O.mstep(pr, np.zeros((37, 28)))
        lse, dS, _ = O.estep_stats(X[rank::WS], post)
        t = torch.from_numpy(np.concatenate([dS.ravel(), [lse.sum()]]))
        dist.all_reduce(t)
        q.put((rank, t.numpy()))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_points_sharded_over_two_ranks_sum_to_the_whole_frame():
    """Eq. 3's statistics and the per-point lse are sums over points, so a
    frame split across ranks needs one all-reduce of Delta S (K x 28) per
    iteration: the reduced sums equal the whole frame's."""
    import multiprocessing as mp
    from oracle import oracle as O
    from paper_2603_08499_gb300 import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_main, args=(r, port, q)) for r in range(WS)]
    for p in procs:
        p.start()
    try:
        out = sorted((q.get(timeout=120) for _ in range(WS)), key=lambda x: x[0])
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    X, pr = synth.c1_workload(seed=51, N=1_001, K=37)
    lse, dS, _ = O.estep_stats(X, O.mstep(pr, np.zeros((37, 28))))
    whole = np.concatenate([dS.ravel(), [lse.sum()]])
    for _, t in out:
        assert np.allclose(t, whole, rtol=1e-12, atol=1e-9 * np.abs(whole).max())


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

"""The N > 1 host path of bench.py on CPU with two gloo ranks: the job time
is the slowest rank's timed region; a batch is partitioned over the ranks by
work and the per-system results are gathered back, covering every system
exactly once."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t_local = [0.8, 1.3][rank]
        v = bench.job_seconds_per_solve(t_local, 5, world, dist, torch, torch.device("cpu"))
        vp = bench.job_seconds_per_solve(t_local, 5, world, dist, torch, torch.device("cpu"), replicas=False)
        # partition 7 systems of uneven work, "solve" the local share (here:
        # a value that identifies the system), gather
        works = [3.0, 8.0, 1.0, 5.0, 5.0, 2.0, 4.0]
        mine = bench.partition(works, world)[rank]
        local = {k: float(10 * k + 1) for k in mine}
        merged = bench.gather_results(local, world, dist)
        dist.barrier()
        q.put((rank, v, vp, mine, merged))
    finally:
        dist.destroy_process_group()


def test_two_rank_partition_and_gather():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = {r: (v, vp, mine, merged) for r, v, vp, mine, merged in (q.get(timeout=10) for _ in range(2))}
    # replicas: slowest rank (1.3 s) over 2 ranks x 5 solves; partition: over 5 solves of one workload
    for r in range(2):
        assert got[r][0] == pytest.approx(1.3 / 10) and got[r][1] == pytest.approx(1.3 / 5)
    # the shares are disjoint, cover all 7 systems, and balance the work
    s0, s1 = set(got[0][2]), set(got[1][2])
    assert not (s0 & s1) and s0 | s1 == set(range(7))
    works = [3.0, 8.0, 1.0, 5.0, 5.0, 2.0, 4.0]
    assert abs(sum(works[i] for i in s0) - sum(works[i] for i in s1)) <= max(works)
    # every rank gets every system's result, each from the rank that solved it
    for r in range(2):
        assert got[r][3] == {k: float(10 * k + 1) for k in range(7)}


def test_single_rank_needs_no_collective():
    import bench
    assert bench.job_seconds_per_solve(2.0, 4, 1, None, torch, None) == pytest.approx(0.5)
    assert bench.gather_results({3: 1.0}, 1, None) == {3: 1.0}

"""The N > 1 host path of bench.py on CPU: two gloo ranks, each with its own
replica of the workload and no collective on the data path; the job time is
the slowest rank's timed region over all ranks' solves."""

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
        dist.barrier()
        q.put((rank, v))
    finally:
        dist.destroy_process_group()


def test_two_rank_job_time_is_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = dict(q.get(timeout=10) for _ in range(2))
    # slowest rank (1.3 s) over 2 ranks x 5 solves, the same on both ranks
    assert got[0] == pytest.approx(1.3 / 10) and got[1] == pytest.approx(1.3 / 10)


def test_single_rank_needs_no_collective():
    import bench
    assert bench.job_seconds_per_solve(2.0, 4, 1, None, torch, None) == pytest.approx(0.5)

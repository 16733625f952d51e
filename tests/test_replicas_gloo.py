"""Multi-process path of the benchmark on CPU: two gloo ranks (replicas, no
data-path collective) agree on the whole-job throughput: every rank's units
over the slowest rank's time."""

import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        ms = [2.0, 3.0][rank]  # the second rank is the slower one
        value, t_max = bench.job_throughput(ms, 1000, world)
        q.put((rank, value, t_max))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_job_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, t_max in res:
        assert t_max == pytest.approx(3.0)
        assert value == pytest.approx(2 * 1000 / 3.0e-3)


def test_single_rank_needs_no_collective():
    import bench
    value, t_max = bench.job_throughput(4.0, 500, 1)
    assert t_max == 4.0 and value == pytest.approx(500 / 4.0e-3)

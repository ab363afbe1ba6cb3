"""The multi-rank measurement path on CPU (gloo, world size 2): the job time
is the slowest rank's, and the job rate counts every rank's units
(replicas of one model; no collective is on the data path)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [120.0, 150.0][rank]  # rank 1 is the slow one
    ms_max = bench.max_over_ranks_on(ms, world, "cpu")
    value = bench.job_throughput(1000, ms_max, world)
    dist.barrier()
    q.put((rank, ms_max, value))
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms_max, value in res:
        assert ms_max == 150.0
        assert abs(value - 2 * 1000 / 0.150) < 1e-6


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks_on(3.5, 1, "cpu") == 3.5
    assert bench.job_throughput(10, 1000.0, 1) == 10.0

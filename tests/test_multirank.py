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


def _lpt_worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2605_30379_gb300 import synth
    shapes = synth.batch_shapes(n=256, seed=0)
    costs = [bench.model_cost(d, N) for d, N in shapes]
    mine = bench.lpt_partition(costs, world)[rank]
    # every rank derives the same partition on its own: gather and compare
    got = [None] * world
    dist.all_gather_object(got, mine)
    ms_max = bench.max_over_ranks_on([100.0, 140.0][rank], world, "cpu")
    dist.barrier()
    q.put((rank, got, sum(costs[i] for i in mine), ms_max))
    dist.destroy_process_group()


def test_batch_lpt_partition_two_ranks_gloo():
    """The 256-model batch split over two ranks by greedy LPT (no collective
    on the data path): the ranks agree on the partition, it covers every model
    exactly once, and the larger load is within Graham's 4/3 - 1/(3m) bound
    of the optimum (bounded below by max(total / m, largest model))."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_lpt_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    import bench
    from paper_2605_30379_gb300 import synth
    costs = [bench.model_cost(d, N) for d, N in synth.batch_shapes(n=256, seed=0)]
    parts = res[0][1]
    assert res[1][1] == parts
    assert sorted(i for p in parts for i in p) == list(range(256))
    loads = [r[2] for r in res]
    opt_lb = max(sum(costs) / 2, max(costs))
    assert max(loads) <= (4 / 3 - 1 / 6) * opt_lb + 1e-6
    assert all(r[3] == 140.0 for r in res)


def test_lpt_partition_small_cases():
    import bench
    assert bench.lpt_partition([5.0, 3.0, 3.0, 2.0, 2.0, 2.0], 2) == [[0, 3, 5], [1, 2, 4]]
    assert bench.lpt_partition([1.0], 3) == [[0], [], []]
    assert bench.lpt_partition([], 2) == [[], []]

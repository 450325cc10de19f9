"""Sharding independent solves over ranks (host side, CPU): the longest-processing-time
partition, and the ranks' timing reductions in world_size-2 gloo process groups (the same
calls the benchmark makes over NCCL)."""
import os
import socket

import pytest

from paper_1012_4307_gb300 import distributed as D

torch = pytest.importorskip("torch")


def test_lpt_partition_covers_every_problem_once():
    sizes = [129, 257, 513, 1025, 1025, 129, 513, 257, 257, 1025, 129, 513, 65]
    costs = [D.solve_cost(n) for n in sizes]
    for nranks in (1, 2, 3, 8, 20):
        parts = D.lpt_partition(costs, nranks)
        assert len(parts) == nranks
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        # LPT bound: no rank exceeds the mean load by more than the largest single job
        loads = [sum(costs[i] for i in p) for p in parts]
        assert max(loads) <= sum(costs) / nranks + max(costs) + 1e-9


def test_lpt_partition_is_deterministic_and_balanced_for_equal_jobs():
    parts = D.lpt_partition([1.0] * 10, 4)
    assert [len(p) for p in parts] == [3, 3, 2, 2]
    assert parts == D.lpt_partition([1.0] * 10, 4)
    with pytest.raises(ValueError):
        D.lpt_partition([1.0], 0)


def test_reductions_without_a_process_group():
    assert D.max_over_ranks(3.5) == 3.5
    assert D.sum_over_ranks(2.0) == 2.0


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, sizes, q):
    import torch.distributed as dist
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        w, r, _ = D.rank_env()
        shard = D.lpt_partition([D.solve_cost(n) for n in sizes], w)[r]
        my_time = 10.0 * (r + 1) + len(shard)
        t = D.max_over_ranks(my_time)
        total = D.sum_over_ranks(sum(sizes[i] ** 2 for i in shard))
        dist.barrier()
        q.put((r, shard, t, total))
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_sharding_and_reductions():
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    sizes = [129, 257, 513, 1025, 1025, 129, 513, 257]
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, sizes, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    shards = [o[1] for o in out]
    assert sorted(shards[0] + shards[1]) == list(range(len(sizes)))
    expect_max = max(10.0 * (r + 1) + len(shards[r]) for r in range(2))
    assert all(o[2] == expect_max for o in out)
    assert all(o[3] == sum(n * n for n in sizes) for o in out)

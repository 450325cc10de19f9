"""Host-side pieces of running many independent solves on several GPUs (one process per GPU).

A single problem does not shard (replicas only).  A batch of independent problems (energies,
right-hand sides, grid sizes) shards by problem: each rank solves the problems assigned to it,
with no data exchange between ranks; the only collectives are a barrier and the max-reduction
of the ranks' timings (the job's time is the slowest rank's).
"""
from __future__ import annotations

import os


def rank_env():
    """(world size, rank, local rank) from the launcher's environment (1, 0, 0 without one)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def solve_cost(n: int, dim: int = 2) -> float:
    """Work estimate of one solve on an n^dim grid: unknowns times an iteration count that grows
    with the wavenumber resolution, taken proportional to n (kh is held fixed as n grows)."""
    return float(n) ** dim * float(n)


def lpt_partition(costs, nranks: int):
    """Longest-processing-time assignment: problems in decreasing cost order, each to the rank
    with the least assigned cost so far (ties: the lowest rank).  Returns one list of problem
    indices per rank, each in decreasing cost order."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * nranks
    parts = [[] for _ in range(nranks)]
    for i in order:
        r = min(range(nranks), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += costs[i]
    return parts


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of value over all ranks of the default process group (value itself when no
    group is initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())

"""Host-side sharding of independent solves over replica ranks.

Independent systems (the batched and serving workloads) need no exchange
between GPUs: each rank runs its own engine on its share of the systems and
the results are gathered on the host.  This module holds that host logic:
a deterministic longest-processing-time assignment of systems to ranks by
an estimated cost, the gathering of per-rank results, and the job-wide
throughput of a timed region (units of all ranks over the slowest rank's
time).  It works with any torch.distributed backend (NCCL on GPUs, gloo on
CPU); nothing here touches a device except through the collectives it is
given.
"""
from __future__ import annotations

import heapq
import math


def solve_cost(n: int, nnz: int, k: int, dim: int = 3) -> float:
    """Estimated cost of a Jacobi-PCG solve of an n-row, nnz-nonzero system
    with k right-hand sides on a stencil of dimension dim: bytes of one
    inner iteration (FP32 values and indices per nonzero, about 44 bytes per
    row and right-hand side) times an iteration count that grows like the
    square root of the condition number, n^(1/dim) for a stencil operator."""
    per_iter = 8.0 * nnz + 44.0 * n * k
    return per_iter * max(1.0, n) ** (1.0 / max(1, dim))


def lpt_assign(costs: list[float], world: int) -> list[int]:
    """Rank of each item: items in decreasing cost (ties by index) go to the
    currently least-loaded rank (ties by rank).  Deterministic, so every
    rank computes the same assignment without communicating; its makespan
    is at most (4/3 - 1/(3 world)) of the optimum (Graham 1969)."""
    if world < 1:
        raise ValueError("world >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    out = [0] * len(costs)
    for i in order:
        load, r = heapq.heappop(heap)
        out[i] = r
        heapq.heappush(heap, (load + costs[i], r))
    return out


def my_share(costs: list[float], rank: int, world: int) -> list[int]:
    """Indices of the items rank `rank` solves, in increasing order."""
    a = lpt_assign(costs, world)
    return [i for i, r in enumerate(a) if r == rank]


def gather_results(local: dict, world: int, group=None) -> dict:
    """Merge every rank's {item index: result} into one dict on every rank
    (torch.distributed.all_gather_object).  An index reported by two ranks
    is an error: the assignment gives each item to exactly one rank."""
    import torch.distributed as dist
    parts = [None] * world
    dist.all_gather_object(parts, local, group=group)
    out = {}
    for p in parts:
        for i, v in p.items():
            if i in out:
                raise RuntimeError(f"item {i} solved by two ranks")
            out[i] = v
    return out


def job_throughput(local_units: float, local_seconds: float, device=None, group=None) -> float:
    """Units processed by all ranks divided by the slowest rank's time."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return local_units / local_seconds
    t = torch.tensor([float(local_units), float(local_seconds)], dtype=torch.float64, device=device)
    units = t[:1].clone()
    secs = t[1:].clone()
    dist.all_reduce(units, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(secs, op=dist.ReduceOp.MAX, group=group)
    if not math.isfinite(float(secs.item())) or float(secs.item()) <= 0.0:
        raise ValueError("timed region must be positive")
    return float(units.item()) / float(secs.item())

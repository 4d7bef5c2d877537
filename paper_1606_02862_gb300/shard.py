"""Sharding of independent boxes over ranks (one process per GPU).

Independent periodic boxes exchange nothing, so a batch of them shards by
box with no collective on the data path: each rank builds one context with
its share and advances it; the only collectives are the timing barrier and
a max-over-ranks of the measured times (and, when wanted, a gather of the
FP64 diagnostics).  A single large box does not shard here (that needs a
domain decomposition with guard exchange); bench.py runs it as replicas.
"""
from __future__ import annotations

import heapq


def box_cost(ncells: int, nparticles: int, particle_weight: float = 1.0) -> float:
    """Work estimate of one box: cells for the field update and particles for
    push + deposit (the particle term dominates)."""
    return float(ncells) + particle_weight * float(nparticles)


def partition(costs, nranks: int):
    """Longest-processing-time greedy assignment: boxes in decreasing cost,
    each to the currently lightest rank.  Returns one sorted list of box
    indices per rank; every box appears exactly once."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    heap = [(0.0, r) for r in range(nranks)]
    heapq.heapify(heap)
    parts = [[] for _ in range(nranks)]
    for i in sorted(range(len(costs)), key=lambda k: (-costs[k], k)):
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(p) for p in parts]


def imbalance(costs, parts) -> float:
    """max rank load / mean rank load (1.0 = perfect)."""
    loads = [sum(costs[i] for i in p) for p in parts]
    mean = sum(loads) / max(len(loads), 1)
    return max(loads) / mean if mean > 0 else 1.0


def max_over_ranks(values, dist=None, device=None):
    """Element-wise maximum of a list of floats over all ranks (identity
    without a process group).  Uses a CPU tensor for gloo, `device` for nccl."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return [float(v) for v in values]
    import torch

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def sum_over_ranks(values, dist=None, device=None):
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return [float(v) for v in values]
    import torch

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return [float(v) for v in t.cpu()]

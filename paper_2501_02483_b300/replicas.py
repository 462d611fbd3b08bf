"""Host-side helpers for running independent replicas on several GPUs.

The library factorizes each matrix on one GPU.  Across GPUs the natural unit
of parallelism is the matrix (Appendix A of the paper runs many independent
factorizations at once): a batch of a hyperparameter sweep or a stream of
requests is split by matrix, each rank factorizes its own matrices with no
collective on the data path, and only small per-matrix results (log-
determinants, residuals, timings) are gathered at the end.  This module holds
that host logic; it works with any torch.distributed backend (NCCL between
GPUs, gloo on CPU for tests).
"""
from __future__ import annotations

__all__ = ["partition_by_cost", "max_over_ranks", "gather_by_index"]


def partition_by_cost(costs, world):
    """Split items with the given costs over ``world`` ranks: largest first,
    each to the rank with the least total so far (ties to the lowest rank).
    Deterministic; returns one ascending index list per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += float(costs[i])
    return [sorted(p) for p in parts]


def max_over_ranks(dist, value, device=None):
    """The maximum of a float over all ranks (the slowest rank's time); the
    value itself when ``dist`` is None or not initialised."""
    if dist is None or not dist.is_initialized():
        return value
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_by_index(dist, local):
    """Merge per-rank {item index: result} dicts into one dict on every rank."""
    if dist is None or not dist.is_initialized():
        return dict(local)
    out = [None] * dist.get_world_size()
    dist.all_gather_object(out, dict(local))
    merged = {}
    for part in out:
        for k, v in part.items():
            if k in merged:
                raise ValueError(f"item {k} came from two ranks")
            merged[k] = v
    return merged

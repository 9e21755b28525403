"""Multi-rank helpers (one process per GPU, torch.distributed).

The path shards by cameras/pixels with no exchange in the forward pass, so a
multi-GPU run is a set of replicas: each rank renders its own seeds or its own
share of the jobs, and only the timing is reduced (max over ranks).  If one
image's samples were split across ranks, the adjoint would need one all-reduce
(sum) of the gradient buffers; ``allreduce_gradients`` is that step.
"""
from __future__ import annotations

from typing import List

import torch
import torch.distributed as dist


def world() -> tuple:
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def rank_seeds(rank: int, base: int = 1000) -> tuple:
    """Forward / backward PCG32 initstates of a rank (distinct across ranks and phases)."""
    return base + 2 * rank, base + 2 * rank + 1


def partition(n_items: int, rank: int, world_size: int) -> List[int]:
    """Round-robin share of items for a rank (every item on exactly one rank)."""
    return list(range(rank, n_items, world_size))


def max_over_ranks(value: float, device="cpu") -> float:
    r, w = world()
    if w == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device="cpu") -> float:
    r, w = world()
    if w == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def allreduce_gradients(grads: List[torch.Tensor]) -> None:
    """Sum gradient buffers over ranks in place (the adjoint's one exchange step)."""
    r, w = world()
    if w == 1:
        return
    for g in grads:
        dist.all_reduce(g, op=dist.ReduceOp.SUM)

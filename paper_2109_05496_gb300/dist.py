"""Multi-process helpers for running independent denoising problems on several
GPUs (one process per GPU). The method has no exchange step between images, so
the only collectives are for measurement: a barrier and a max over ranks of the
timed region. Images of uneven sizes are spread over ranks by cost.
"""
from __future__ import annotations

import heapq
from typing import List, Sequence, Tuple

import torch


def shard_range(count: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous, balanced [start, stop) of `count` units for `rank`."""
    if world <= 0 or not 0 <= rank < world or count < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(count, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def shard_by_cost(costs: Sequence[float], world: int) -> List[List[int]]:
    """Longest-processing-time assignment of units (e.g. images, cost = pixels)
    to `world` ranks; every rank gets a deterministic list of unit indices."""
    if world <= 0:
        raise ValueError("world must be positive")
    heap = [(0.0, r) for r in range(world)]
    out: List[List[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    for lst in out:
        lst.sort()
    return out


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of a scalar over all ranks (identity without a process group)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    if device is None:
        device = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_value(units_per_rank: float, max_ms: float, world: int) -> float:
    """Whole-job throughput when every rank processes the same number of units."""
    return world * units_per_rank / (max_ms * 1e-3)

"""Multi-GPU layout of the hot path: independent systems per rank.

The WaveHoltz solves of different shots and frequencies are independent
problems, so they shard across ranks with no data-path collective.  Only the
bookkeeping is collective: the slowest rank's time and the total work.  (One
large system would instead be split into slabs with a halo exchange once per
time level and one FP64 allreduce per CG iteration; that layout is not built
because every machine this runs on gives a process one GPU.)
"""
from __future__ import annotations

from typing import List, Sequence


def shard(n_items: int, rank: int, world: int) -> List[int]:
    """Round-robin assignment of item indices to ``rank`` of ``world``."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("rank must lie in [0, world)")
    return list(range(rank, n_items, world))


def shot_positions(length: float, n_shots: int) -> List[float]:
    """Evenly spaced shot positions strictly inside [0, length]."""
    return [length * (k + 1) / (n_shots + 1) for k in range(n_shots)]


def reduce_job(elapsed_s: float, work_units: float, device=None):
    """(max elapsed over ranks, total work over ranks); identity without a
    process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return elapsed_s, work_units
    t = torch.tensor([float(elapsed_s)], dtype=torch.float64, device=device)
    w = torch.tensor([float(work_units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    return float(t.item()), float(w.item())


def gather_results(local: Sequence, n_items: int, rank: int, world: int):
    """Reassemble per-item results computed by ``shard`` on every rank into
    item order (every rank receives the full list)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or world == 1:
        return list(local)
    parts = [None] * world
    dist.all_gather_object(parts, list(local))
    out = [None] * n_items
    for r in range(world):
        for k, idx in enumerate(shard(n_items, r, world)):
            out[idx] = parts[r][k]
    return out

"""Multi-GPU layout of the batched transform: every signal is independent,
so N ranks each transform their own batch (weak scaling) with the plan
replicated and no exchange on the data path.  Only the benchmark's timing
crosses ranks: the step time is the maximum over ranks."""
from __future__ import annotations


def rank_seed(base_seed: int, rank: int) -> int:
    """Signal seed of a rank's own batch (distinct per rank, reproducible)."""
    return base_seed + 7919 * rank


def shard_rows(total: int, rank: int, world: int):
    """[start, stop) of rank's share when one global batch is split by rows."""
    per = -(-total // world)
    start = min(total, rank * per)
    return start, min(total, start + per)


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Largest value over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())

"""Multi-rank host logic (one process per GPU).

The index partitions rows exactly like the paper's machines (Sec. 3): rank r
owns the contiguous row range [r*n, (r+1)*n) of the global dataset, builds its
own index with the shared seed and answers its own query batch.  Nothing is
exchanged on the data path (weak scaling); the only collectives are the
timing barrier and the max-over-ranks reduction of the step time.
"""
from __future__ import annotations


def rank_rows(rank: int, world: int, rows_per_rank: int) -> tuple[int, int]:
    """(first global row, rows) of this rank's partition."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return rank * rows_per_rank, rows_per_rank


def max_over_ranks(values: list[float], device=None) -> list[float]:
    """Element-wise max of per-rank timings (identity when not distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(values)
    t = torch.tensor(values, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_throughput(units_per_rank: int, world: int, max_seconds: float) -> float:
    """Whole-job rate: every rank's units over the slowest rank's time."""
    return units_per_rank * world / max_seconds

"""Replica bookkeeping for runs on several GPUs.

The (sample pair, tau) units of the self-energy are independent, so N GPUs
run N independent replicas, one process each: every rank draws its own
seeds, there is no collective on the data path, and the job's throughput is
the units of all ranks over the slowest rank's time (weak scaling).  Only the
timing uses a collective (a max over ranks).
"""
from __future__ import annotations

RANK_SEED_STRIDE = 1_000_000


def rank_seed(rank: int, step: int) -> int:
    """Seed of step `step` on rank `rank` (disjoint streams across ranks)."""
    if step < 0 or step >= RANK_SEED_STRIDE:
        raise ValueError("step out of range")
    return rank * RANK_SEED_STRIDE + step


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over the ranks of the default process group
    (the value itself when no group is initialised)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_step: int, steps: int, world: int, seconds_max: float) -> float:
    """Whole-job units per second: all ranks' units over the slowest time."""
    if seconds_max <= 0:
        raise ValueError("time must be positive")
    return units_per_step * steps * world / seconds_max

"""Replica bookkeeping for one process per GPU.

Particles are independent (no space charge), so N GPUs track N independent
ensembles, each rank its own seeded ensemble of the same size (weak scaling);
nothing on the data path is exchanged.  Only the timings are reduced: the
job's time is the slowest rank's, and the job's rate is the units all ranks
processed over that time.
"""
from __future__ import annotations


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of a rank's ensemble: distinct per rank, reproducible."""
    return int(base_seed) + int(rank)


def max_over_ranks(value: float, dist=None, device: str = "cpu") -> float:
    """Maximum of a per-rank scalar over all ranks (identity without a process group)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank: float, world: int, t_max: float) -> float:
    """Whole-job rate: units processed by all ranks over the slowest rank's time."""
    if not t_max > 0:
        raise ValueError("t_max must be positive")
    return float(units_per_rank) * int(world) / float(t_max)

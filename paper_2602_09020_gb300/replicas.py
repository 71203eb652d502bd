"""Replica bookkeeping for multi-process benchmark runs (one process per GPU).

The statevector does not shard on one-GPU machines, so N processes run N
independent replicas of the same workload.  The whole-job figure is the work
all ranks did divided by the slowest rank's time; these helpers do that
reduction with torch.distributed (any backend: NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import torch


def max_over_ranks(value: float, dist=None, device: str = "cpu") -> float:
    """Maximum of a per-rank float over all ranks (identity without a group)."""
    if dist is None or not dist.is_initialized():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, seconds_max: float, world: int) -> float:
    """Units per second for the whole job: every rank's units over the slowest rank's time."""
    if seconds_max <= 0:
        raise ValueError("time must be positive")
    return world * units_per_rank / seconds_max

"""Host logic of multi-GPU runs: independent replicas, one process per GPU.

Sub-queries and rows are independent (the paper's sub-query touches one
table; there is no exchange step), so N GPUs run N replicas of the same
workload on their own seeded tables (weak scaling) with no data-path
collective.  The only collectives are the measurement's: a barrier on both
sides of the timed region and the maximum of the ranks' times.  Works with
the nccl backend (CUDA tensors) and with gloo (CPU tensors, used by the
tests).
"""
from __future__ import annotations

import os
from typing import Optional, Tuple

import torch


def env_rank() -> Tuple[int, int, int]:
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def table_seed(rank: int, base: int = 2) -> int:
    """Seed of the table a rank scans (distinct tables, same distribution)."""
    return base + rank


def max_over_ranks(ms: float, dist=None, device: Optional[torch.device] = None) -> float:
    """The slowest rank's time (the job ends when the last rank ends)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(ms)
    x = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(x, op=dist.ReduceOp.MAX)
    return float(x.item())


def job_value(units_per_rank: int, world: int, ms: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest time."""
    return units_per_rank * world / (ms / 1e3)

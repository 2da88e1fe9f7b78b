"""Multi-GPU bookkeeping for replicated runs.

Within one mapping or tracking iteration the hot path does not shard across GPUs here:
``bench.py --gpus N`` runs one independent replica per rank (one process per GPU, weak
scaling). Each rank times its own steps between barriers; the job's time is the maximum
over ranks and its throughput is the work of all ranks divided by that time.
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def rank_and_world() -> tuple[int, int]:
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def barrier():
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def max_over_ranks(x: float, device=None) -> float:
    """Maximum of a per-rank scalar over all ranks (identity when not distributed)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank: float, world: int, max_seconds: float) -> float:
    """Units processed by all ranks per second of the slowest rank."""
    return units_per_rank * world / max_seconds

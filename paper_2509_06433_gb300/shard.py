"""A mapping window's views sharded over ranks (one process per GPU).

The K key-frames of a window share one Gaussian set: every rank holds the whole map, renders
and differentiates its contiguous share of the views (its own Rasterizer with K_rank views),
and the exchange step is the sum of the per-Gaussian gradients over ranks — one all-reduce of
one packed buffer (means, log-scales, quaternions, opacity logits, colours) — plus an all-gather
of the per-view pose gradients, so that every rank ends with what a single K-view launch would
have produced (up to the summation order). The sums run on whatever backend the process group
has (NCCL between GPUs, gloo on the host).
"""
from __future__ import annotations

import torch
import torch.distributed as dist

NAMES = ("means", "log_scales", "quats", "opacity_logits", "rgb")


def view_range(K: int, rank: int, world: int) -> tuple[int, int]:
    """The contiguous views [start, stop) of `rank`: the first K % world ranks take one more."""
    base, extra = divmod(K, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def allreduce_gaussian_grads(grads: dict, group=None) -> dict:
    """Sums the five per-Gaussian gradient tensors of `grads` over the ranks, in place, with one
    all-reduce of a packed buffer. Returns `grads`."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return grads
    parts = [grads[k].reshape(-1) for k in NAMES]
    flat = torch.cat(parts)
    dist.all_reduce(flat, op=dist.ReduceOp.SUM, group=group)
    off = 0
    for k, p in zip(NAMES, parts):
        grads[k].copy_(flat[off:off + p.numel()].view_as(grads[k]))
        off += p.numel()
    return grads


def gather_pose_grads(pose_local: torch.Tensor, K: int, group=None) -> torch.Tensor:
    """The [K, 6] pose gradients of all views, from each rank's [K_rank, 6] (its view_range)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return pose_local
    world = dist.get_world_size(group)
    cap = -(-K // world)
    padded = torch.zeros((cap, 6), dtype=pose_local.dtype, device=pose_local.device)
    padded[:pose_local.shape[0]] = pose_local
    out = [torch.empty_like(padded) for _ in range(world)]
    dist.all_gather(out, padded, group=group)
    rows = []
    for r in range(world):
        a, b = view_range(K, r, world)
        rows.append(out[r][:b - a])
    return torch.cat(rows)

"""Data parallelism over rays (host side).

Rays are independent, so a batch splits into contiguous per-rank shards with
no exchange in the forward pass; the backward pass has exactly one exchange:
the per-rank surfel gradients are summed (one all-reduce per gradient
tensor). Works with any torch.distributed backend (NCCL on GPUs, gloo on
CPU)."""
from __future__ import annotations

import torch
import torch.distributed as dist


def ray_shard(n_rays: int, world: int, rank: int) -> slice:
    """Contiguous shard of rank `rank` (sizes differ by at most one)."""
    if world <= 0 or not 0 <= rank < world:
        raise ValueError("bad world/rank")
    base, extra = divmod(n_rays, world)
    start = rank * base + min(rank, extra)
    return slice(start, start + base + (1 if rank < extra else 0))


def allreduce_grads(grads: dict) -> dict:
    """Sum the surfel gradients of all ranks in place (no-op on one rank)."""
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        for k in sorted(grads):
            dist.all_reduce(grads[k], op=dist.ReduceOp.SUM)
    return grads

"""Replicas: one process per GPU, each holding the whole database and index.

Queries are independent, so a batch is split into contiguous shards, one per
rank, with no collective on the data path.  The only communication is
host-level bookkeeping: the slowest rank's time (the job's time) and, when a
caller wants every answer on one rank, a gather of the shards' results.
"""
from __future__ import annotations


def shard(n_total: int, world: int, rank: int):
    """Contiguous [lo, hi) share of n_total queries for `rank` (sizes differ by at most 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must be in [0, world)")
    base, extra = divmod(n_total, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of `value` over all ranks (the job finishes with its slowest rank)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_rows(local, n_total: int, device=None):
    """Concatenate every rank's rows (in rank order) on every rank."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return local
    world = dist.get_world_size()
    sizes = [shard(n_total, world, r)[1] - shard(n_total, world, r)[0] for r in range(world)]
    width = local.shape[1:]
    maxn = max(sizes)
    pad = torch.zeros((maxn,) + tuple(width), dtype=local.dtype, device=device)
    pad[: local.shape[0]] = local
    parts = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    return torch.cat([p[:s] for p, s in zip(parts, sizes)])

"""Several GPUs, one process each.

Replicas: every rank holds the whole database and index and answers its own
contiguous shard of the queries, with no collective on the data path; the
only communication is host-level bookkeeping (the slowest rank's time, and a
gather of the shards' results when a caller wants them on one rank).

Database shards: every rank holds one contiguous id range of the database
and its index, and answers every query over its range.  The exchange step is
one all-gather of the ranks' (nq, k) answers; mih_merge_topk (a library
kernel) then merges them exactly, since the ranges partition the database
and (distance, id) is a total order.
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


def db_shard(n: int, world: int, rank: int):
    """Contiguous id range [lo, hi) of an n-code database held by `rank`."""
    return shard(n, world, rank)


def all_gather_parts(ids, dist):
    """Every rank's (nq, k) answers stacked in rank order: (world, nq, k) each."""
    import torch
    import torch.distributed as dist_

    if not (dist_.is_available() and dist_.is_initialized()) or dist_.get_world_size() == 1:
        return ids.unsqueeze(0).contiguous(), dist.unsqueeze(0).contiguous()
    world = dist_.get_world_size()
    pi = [torch.empty_like(ids) for _ in range(world)]
    pd = [torch.empty_like(dist) for _ in range(world)]
    dist_.all_gather(pi, ids.contiguous())
    dist_.all_gather(pd, dist.contiguous())
    return torch.stack(pi).contiguous(), torch.stack(pd).contiguous()


def knn_db_sharded(index, queries, k: int, n_total: int, stream=None):
    """Exact k-NN over the whole database from this rank's id range: the
    rank's own mih_knn, the all-gather of every rank's answer and the exact
    merge (mih_merge_topk).  Every rank returns the same {"ids", "dist"}."""
    import torch.distributed as dist_

    from . import mih_knn, mih_merge_topk

    world = dist_.get_world_size() if (dist_.is_available() and dist_.is_initialized()) else 1
    local = mih_knn(index, queries, k, stream=stream)
    pi, pd = all_gather_parts(local["ids"], local["dist"])
    bases = [db_shard(n_total, world, r)[0] for r in range(world)]
    return mih_merge_topk(pi, pd, bases, k, stream=stream)

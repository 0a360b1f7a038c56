"""Sharding of a scan across ranks (one process per GPU).

Scan points are independent (each pair is registered, fitted and solved on
its own), so the data path has no collective: every rank takes a contiguous
range of points, and only the per-pair results (F, R_finite, status) are
gathered at the end.  These helpers hold that host-side logic; they work with
any torch.distributed backend (NCCL between GPUs, gloo on CPU for tests).
"""
from __future__ import annotations


def shard_range(n_total: int, rank: int, world: int) -> range:
    """Contiguous, balanced range of scan points of `rank` (the first n_total % world ranks get one more)."""
    if world < 1 or not 0 <= rank < world or n_total < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_total, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a float over all ranks (the step time of the slowest rank)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_results(local: dict, n_total: int, device=None) -> dict | None:
    """Concatenate each rank's per-pair result tensors (first dimension = its shard) on rank 0.

    Shards may differ in length by one; they are padded to the largest shard for the
    collective and trimmed after.  Returns the full-scan tensors on rank 0, None elsewhere."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized() or dist.get_world_size() == 1:
        return {k: v for k, v in local.items()}
    world, rank = dist.get_world_size(), dist.get_rank()
    sizes = [len(shard_range(n_total, r, world)) for r in range(world)]
    m = max(sizes)
    out = {}
    for k in sorted(local):
        v = local[k]
        pad = torch.zeros((m,) + tuple(v.shape[1:]), dtype=v.dtype, device=device if device is not None else v.device)
        pad[:v.shape[0]] = v
        parts = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(parts, pad)
        if rank == 0:
            out[k] = torch.cat([p[:s] for p, s in zip(parts, sizes)])
    return out if rank == 0 else None

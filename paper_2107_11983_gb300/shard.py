"""Splitting a walk batch over ranks (one process per GPU, graph replicated).

A walk depends only on (seed, walk index), so ranks need no exchange: each
rank runs its own range of walk indices through ``walk_offset`` and the
union of the ranks' outputs equals the single-process result.
"""
from __future__ import annotations


def weak_shard(walks_per_rank: int, rank: int) -> int:
    """walk_offset of rank's batch when every rank runs walks_per_rank walks."""
    if walks_per_rank < 0 or rank < 0:
        raise ValueError("negative size or rank")
    return rank * walks_per_rank


def strong_shard(n_walks: int, rank: int, world: int) -> tuple:
    """Contiguous [lo, hi) of n_walks for rank out of world (sizes differ by at most one)."""
    if world < 1 or not 0 <= rank < world or n_walks < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_walks, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return lo, hi

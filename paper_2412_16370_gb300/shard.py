"""Splitting one count across ranks (one process per GPU).

Counts are additive under concatenation of whole words (Section 4, step 1
and its footnote: counts are added into C, so non-contiguous pieces of one
input can be counted into one counter array).  A byte range is therefore cut
into per-rank shards whose boundaries are multiples of 64 bytes from the
start: every shard starts on a word boundary for every w <= 64 (and on the
same 16-byte phase as the whole), so each rank counts its shard with the
single-array entry point and one sum of w counters per rank completes it.
"""
from __future__ import annotations

ALIGN = 64


def shard_range(nbytes: int, rank: int, world: int, align: int = ALIGN) -> tuple[int, int]:
    """Byte range ``[lo, hi)`` of ``rank``'s shard of ``nbytes`` bytes."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need 0 <= rank < world")
    if align < 1 or align % 8:
        raise ValueError("align must be a positive multiple of 8")
    units = (nbytes + align - 1) // align
    per, extra = divmod(units, world)
    u0 = rank * per + min(rank, extra)
    u1 = u0 + per + (1 if rank < extra else 0)
    return min(nbytes, u0 * align), min(nbytes, u1 * align)


def all_ranks_ranges(nbytes: int, world: int, align: int = ALIGN) -> list[tuple[int, int]]:
    return [shard_range(nbytes, r, world, align) for r in range(world)]


def sum_counts(counts, group=None):
    """All-reduce (sum) one rank's counters over the process group, in place."""
    import torch.distributed as dist
    dist.all_reduce(counts, op=dist.ReduceOp.SUM, group=group)
    return counts

"""Partition of independent work over the ranks of a multi-GPU job (one process per GPU).

A single instance does not shard (each Tabu iteration waits on the previous one's
move), but batches and request streams are independent instances: every rank takes
its own part and solves it alone, with no collective on the data path. Only the
host-side gather of results and timings crosses ranks.

  contiguous(n, rank, world)  the rank's block [lo, hi) of n items: sizes differ by at
                              most one, blocks are in rank order and cover 0..n-1 once.
  strided(n, rank, world)     items rank, rank + world, ...: a request stream dealt
                              round-robin (every rank sees 1/world of the arrival rate).
"""
from __future__ import annotations


def contiguous(n: int, rank: int, world: int) -> tuple[int, int]:
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("need n >= 0 and 0 <= rank < world")
    q, r = divmod(n, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def strided(n: int, rank: int, world: int) -> range:
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("need n >= 0 and 0 <= rank < world")
    return range(rank, n, world)

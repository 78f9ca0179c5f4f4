"""Replica sharding of one instance across processes (one GPU each).

The subproblems of the l-mers of S_1 are independent (Section 2.3), so N replicas can
split them into N contiguous ranges, solve their range with pms_opts.x_begin/x_end, and
merge the sorted motif sets.  The merge is the only exchange the method needs (the
paper's workers send their motifs to the scheduler at the end); it is a host-side
all-gather of sorted lists, not a device collective.
"""

from __future__ import annotations

import heapq
from typing import Callable, Sequence


def shard_ranges(L: int, world: int) -> list[tuple[int, int]]:
    """Contiguous ranges of x in [0, L) for `world` replicas, sizes differing by <= 1."""
    if world < 1:
        raise ValueError("world must be >= 1")
    base, extra = divmod(L, world)
    out, lo = [], 0
    for r in range(world):
        hi = lo + base + (1 if r < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


def merge_sorted(parts: Sequence[Sequence[str]], alphabet: str) -> list[str]:
    """Union of sorted motif lists, sorted in the alphabet's order, each motif once."""
    rank = {c: i for i, c in enumerate(alphabet)}
    key = (lambda s: tuple(rank[c] for c in s))
    out: list[str] = []
    for m in heapq.merge(*parts, key=key):
        if not out or out[-1] != m:
            out.append(m)
    return out


def solve_sharded(solve_range: Callable[[int, int], list[str]], L: int, alphabet: str,
                  rank: int, world: int, group=None) -> list[str]:
    """Solve this rank's range with `solve_range(x_begin, x_end)` and return the merged
    set on every rank (torch.distributed all_gather_object over `group`)."""
    lo, hi = shard_ranges(L, world)[rank]
    mine = solve_range(lo, hi) if hi > lo else []
    if world == 1:
        return mine
    import torch.distributed as dist
    parts: list = [None] * world
    dist.all_gather_object(parts, mine, group=group)
    return merge_sorted(parts, alphabet)

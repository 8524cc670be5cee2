"""Query sharding across ranks (one process per GPU).

The hot path has no exchange step: every query (and every volume pixel) is independent
and its random numbers are keyed by its global id, so a rank evaluates a contiguous
range of ids with ``id_base`` set to the range start and the union of the shards equals
the single-GPU result bit for bit.  Strong scaling splits one batch; weak scaling gives
every rank its own batch of the same size with disjoint id ranges.
"""
from __future__ import annotations


def shard(n: int, rank: int, world: int) -> tuple[int, int]:
    """(begin, count) of rank's contiguous share of n items (first n % world ranks get one more)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(n, world)
    begin = rank * base + min(rank, extra)
    return begin, base + (1 if rank < extra else 0)


def weak_id_base(rank: int, per_rank: int) -> int:
    """First query id of rank's own batch under weak scaling."""
    return rank * per_rank

"""Sharding across ranks (one process per GPU).

The lookup path has no exchange step: every query (and every volume pixel) is independent
and its random numbers are keyed by its global id, so a rank evaluates a contiguous
range of ids with ``id_base`` set to the range start and the union of the shards equals
the single-GPU result bit for bit.  Strong scaling splits one batch; weak scaling gives
every rank its own batch of the same size with disjoint id ranges.

Training of the learned form has one exchange step per optimiser step: the ranks'
gradients of their shares of the batch are summed (all-reduce) before the identical Adam
updates of the replicas (``dp_train``).
"""
from __future__ import annotations

from typing import Callable


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


def dp_train(steps: int, batch: int, rank: int, world: int, grad: Callable[[int, int, int], None],
             allreduce: Callable[[], None], adam: Callable[[int], None]) -> None:
    """Data-parallel optimiser loop of one rank.  For k = 0 .. steps-1: grad(k, first, count)
    computes this rank's share of step k's batch (gradients normalised by the whole batch),
    allreduce() sums the gradient arrays over the ranks in place, adam(k) applies step k.
    Every rank runs the same sequence of collectives (one per step)."""
    first, count = shard(batch, rank, world)
    for k in range(steps):
        grad(k, first, count)
        if world > 1:
            allreduce()
        adam(k)

"""Assignment of independent simulation instances to ranks (one process per GPU).

The batched workload is a set of independent subvolumes: they share nothing during the time loop,
so ranks split the instances and run them with no collective on the data path.  Instances are
dealt greedily by node count (largest first, to the rank with the fewest nodes so far, ties to
the lowest rank), which balances uneven sizes and is the same on every rank.
"""
from __future__ import annotations


def shard_instances(sizes, world: int, rank: int) -> list[int]:
    """Indices of the instances rank `rank` of `world` runs, given every instance's node count."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need world >= 1 and 0 <= rank < world")
    load = [0] * world
    owner = [0] * len(sizes)
    for i in sorted(range(len(sizes)), key=lambda k: (-int(sizes[k]), k)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += int(sizes[i])
    return [i for i in range(len(sizes)) if owner[i] == rank]


def rank_loads(sizes, world: int) -> list[int]:
    return [sum(int(sizes[i]) for i in shard_instances(sizes, world, r)) for r in range(world)]

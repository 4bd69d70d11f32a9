"""Partition of a batched replica set over ranks (Sec. 4.2: independent
systems advanced together; one process per GPU).

The replicas are independent, so a job over several GPUs gives each rank a
share of them and needs no data-path collective: each rank builds and
advances its own replicas with the batched engine, the job takes as long as
its slowest rank, and its rate counts every rank's particles.  A replica's
initial state depends only on its own seed, so a rank generates exactly the
replicas a single process would.

The shares balance the particle count (the work of a step is about
proportional to it): largest replica first, each to the rank with the fewest
particles so far (ties to the lower rank).  The split is a pure function of
the sizes and the number of ranks, so every rank computes the same one
without communication.
"""
from __future__ import annotations


def split_replicas(sizes, world: int) -> list[list[int]]:
    """Replica indices of each of `world` ranks (each list ascending)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    shares: list[list[int]] = [[] for _ in range(world)]
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        shares[r].append(i)
        load[r] += int(sizes[i])
    return [sorted(s) for s in shares]

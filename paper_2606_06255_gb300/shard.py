"""Sharding independent clouds over ranks (one process per GPU).

Clouds are independent units of work, so a multi-GPU run needs no
collective on the data path: every rank computes the same deterministic
assignment, samples its own clouds, and only the host gathers results.  The
assignment is longest-processing-time first on the per-cloud work N_b * M_b
(the plain FPS cost; the pruned loop's cost grows with it too), ties broken
by cloud index, each cloud going to the least-loaded rank (lowest rank on
ties).
"""

from __future__ import annotations


def assign(sizes, ms, world: int):
    """List of cloud-index lists, one per rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    work = [int(n) * int(m) for n, m in zip(sizes, ms)]
    order = sorted(range(len(work)), key=lambda b: (-work[b], b))
    load = [0] * world
    shards = [[] for _ in range(world)]
    for b in order:
        r = min(range(world), key=lambda k: (load[k], k))
        shards[r].append(b)
        load[r] += work[b]
    return [sorted(s) for s in shards]


def my_clouds(sizes, ms, world: int, rank: int):
    return assign(sizes, ms, world)[rank]

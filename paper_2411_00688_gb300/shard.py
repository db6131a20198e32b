"""Problem-level split of a batch of independent solves over ranks (one GPU each).

The problems of a batch share no data and each one's coins depend only on its own
seed, so ranks can solve disjoint subsets with no exchange at all; the split only
has to balance the work.  Longest-processing-time-first greedy (Graham, 1969):
problems in decreasing cost order, each to the rank with the least work so far,
which keeps the busiest rank within 4/3 of the optimum makespan.  Every rank
computes the same split from the same costs, so no communication is needed to
agree on it.
"""

from __future__ import annotations


def lpt_shards(costs, world: int):
    """Indices of the problems each rank solves (a list per rank, each in
    increasing index order), for per-problem costs ``costs``."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    shards = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        shards[r].append(i)
        load[r] += float(costs[i])
    return [sorted(s) for s in shards]

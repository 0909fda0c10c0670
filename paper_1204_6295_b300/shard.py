"""Assignment of independent registration pairs to ranks (one GPU per rank).

The pairs of the batched form are independent problems: their data paths
exchange nothing, so sharding them across GPUs needs no collective beyond the
final gather of results.  Each rank takes its share by the
longest-processing-time rule: pairs in decreasing order of work (voxel
iterations of the whole schedule), each to the rank with the least work so
far.  The slowest rank then carries at most (4/3 - 1/(3m)) times the optimal
makespan on m ranks (Graham's bound for this rule).  The rule is
deterministic, so every rank computes the same assignment on its own.
"""
from __future__ import annotations


def lpt_assign(loads, nranks):
    """Indices of the pairs each rank runs, [[...] per rank], by decreasing load.

    Ties between pairs go to the lower index first, ties between ranks to the
    lower rank, so the result depends on the loads only.
    """
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    order = sorted(range(len(loads)), key=lambda i: (-loads[i], i))
    share = [[] for _ in range(nranks)]
    total = [0] * nranks
    for i in order:
        r = min(range(nranks), key=lambda k: (total[k], k))
        share[r].append(i)
        total[r] += loads[i]
    return [sorted(s) for s in share]


def rank_loads(loads, share):
    """Work per rank for an assignment."""
    return [sum(loads[i] for i in s) for s in share]

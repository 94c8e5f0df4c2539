"""Partition of a batch of graphs over ranks (Sec. 2 "Batched processing": graphs in a
batch are independent units, their disjoint union renders each graph on its own).

Every rank calls ``partition`` with the same costs and gets the same answer, so ranks
agree on who renders what without exchanging anything; each rank then plans and
renders the union of its own graphs and no collective runs on the data path.
"""


def partition(costs, world):
    """Graph indices per rank, balanced by cost (e.g. nodes x samples): longest
    processing time first, each graph to the rank with the least cost so far (ties to the
    lowest rank), each rank's list in ascending graph order.  Deterministic.  The largest
    rank total is at most 4/3 of the optimum (Graham's bound) and at most the mean plus
    the largest single cost."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda k: (-costs[k], k))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda j: (load[j], j))
        parts[r].append(k)
        load[r] += costs[k]
    return [sorted(p) for p in parts]


def rows_of(graphs, ks, tables):
    """The parameter rows of graphs ks (in that order) from tables over the whole batch
    (rows graph-major in batch order, as ``synth.union_params`` lays them out)."""
    import numpy as np
    out = {}
    for t, tab in tables.items():
        starts, r = [], 0
        for g in graphs:
            starts.append(r)
            r += g.count(t)
        parts = [tab[starts[k]:starts[k] + graphs[k].count(t)] for k in ks if graphs[k].count(t)]
        if parts:
            out[t] = np.ascontiguousarray(np.concatenate(parts))
    return out

"""Small random DAGs for the scheduler and render tests."""
import numpy as np

import synth
from synth import Graph, I, O, M, G, S, E, C


def random_dag(rng, n_inputs=3, n_mid=8, n_outputs=1, kinds=(M, G, S, E, C), p_edge=0.3,
               multi=True):
    """Inputs first, then processing nodes in a random topological order, then outputs.
    Every non-input gets at least one predecessor; outputs have no successors."""
    g = Graph()
    ins = [g.add(I) for _ in range(n_inputs)]
    mids = []
    for _ in range(n_mid):
        v = g.add(int(kinds[int(rng.integers(0, len(kinds)))]))
        cands = ins + mids
        k = int(rng.integers(1, min(3, len(cands)) + 1))
        for s in rng.choice(cands, size=k, replace=False):
            g.connect(int(s), v)
        if multi and rng.random() < 0.1:
            g.connect(int(cands[int(rng.integers(0, len(cands)))]), v)
        mids.append(v)
    sinks = [v for v in mids if not any(s == v for s, _ in g.edges)]
    outs = [g.add(O) for _ in range(n_outputs)]
    for j, v in enumerate(sinks):
        g.connect(v, outs[j % n_outputs])
    for o in outs:
        if not any(d == o for _, d in g.edges):
            g.connect(mids[-1] if mids else ins[0], o)
    return g


def permute_graph(g, perm):
    """Relabel node v as perm[v]; returns the new Graph."""
    n = g.n_nodes
    types = [0] * n
    for v in range(n):
        types[perm[v]] = g.types[v]
    h = Graph(types=types, edges=[(perm[s], perm[d]) for s, d in g.edges], ports=list(g.ports))
    return h


def n_out_ports(t):
    return 2 if t == synth.P else 0 if t == O else 1


def n_in_ports(t):
    return 0 if t == I else 2 if t in (synth.J, synth.K) else 1


def random_mimo_dag(rng, n_inputs=3, n_mid=10, n_outputs=1, kinds=None):
    """Like ``random_dag`` with multi-port nodes: every input port of a node gets 1-2
    edges from random earlier (node, output port) pairs; output ports nobody reads feed
    the graph outputs."""
    kinds = kinds or (M, G, E, C, synth.P, synth.J, synth.K)
    g = Graph()
    ins = [g.add(I) for _ in range(n_inputs)]
    mids = []
    for _ in range(n_mid):
        t = int(kinds[int(rng.integers(0, len(kinds)))])
        v = g.add(t)
        cands = ins + mids
        for l in range(n_in_ports(t)):
            for _ in range(int(rng.integers(1, 3))):
                s = int(cands[int(rng.integers(0, len(cands)))])
                g.connect(s, v, int(rng.integers(0, n_out_ports(g.types[s]))), l)
        mids.append(v)
    used = {(s, k) for (s, d), (k, l) in zip(g.edges, g.ports)}
    outs = [g.add(O) for _ in range(n_outputs)]
    j = 0
    for v in mids:
        for k in range(n_out_ports(g.types[v])):
            if (v, k) not in used:
                g.connect(v, outs[j % n_outputs], k, 0)
                j += 1
    for o in outs:
        if not any(d == o for _, d in g.edges):
            g.connect(mids[-1] if mids else ins[0], o)
    return g

"""Seeded synthetic mixing-console graphs.

A graph is a node-type list and an edge list ``(src, dst)`` in insertion order
(multi-edges allowed), the tensor form of Sec. 2 "Graph representations"
(T_V and E), with the edge types T_E as ``ports[e] = (output k, input l)`` (all
(0, 0) unless a multi-port node is connected).  The builders only draw structure;
scheduling and rendering live elsewhere.
"""
from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

from .types import I, O, M, G, S, E, C, D, R, N


@dataclass
class Graph:
    types: List[int] = field(default_factory=list)
    edges: List[Tuple[int, int]] = field(default_factory=list)
    ports: List[Tuple[int, int]] = field(default_factory=list)

    def __post_init__(self):
        if len(self.ports) != len(self.edges):   # built from (types, edges) alone
            self.ports = [(0, 0)] * len(self.edges)

    # builder calls named after the paper's API (Fig. 2a)
    def add(self, t: int) -> int:
        self.types.append(int(t))
        return len(self.types) - 1

    def add_serial_chain(self, ts):
        ids = [self.add(t) for t in ts]
        for a, b in zip(ids[:-1], ids[1:]):
            self.connect(a, b)
        return ids[0], ids[-1]

    def connect(self, src: int, dst: int, out_port: int = 0, in_port: int = 0):
        self.edges.append((int(src), int(dst)))
        self.ports.append((int(out_port), int(in_port)))

    @property
    def has_ports(self):
        return any(p != (0, 0) for p in self.ports)

    @property
    def n_nodes(self):
        return len(self.types)

    def count(self, t):
        return sum(1 for x in self.types if x == t)


def _partition(rng, items, lo=2, hi=8):
    """Split ``items`` in order into groups of size U{lo..hi}; a leftover
    single item joins the previous group."""
    groups, k = [], 0
    n = len(items)
    if n <= 1:
        return [list(items)] if n else []
    while k < n:
        sz = int(rng.integers(lo, hi + 1))
        grp = items[k:k + sz]
        k += sz
        if len(grp) == 1 and groups:
            groups[-1].extend(grp)
        else:
            groups.append(list(grp))
    return groups


def _subgroups(rng, g: Graph, heads, levels):
    """Nest ``heads`` into ``levels`` levels of mix nodes, then one output."""
    cur = list(heads)
    for _ in range(levels):
        if len(cur) <= 1:
            break
        nxt = []
        for grp in _partition(rng, cur):
            mid = g.add(M)
            for src in grp:
                g.connect(src, mid)
            nxt.append(mid)
        cur = nxt
    out = g.add(O)
    for src in cur:
        g.connect(src, out)
    return g


def console_cfg1() -> Graph:
    """8 tracks i->g->e->c; tracks 0-3 to bus m0, 4-7 to bus m1; both to o.
    35 nodes, 34 edges."""
    g = Graph()
    ends = []
    for _ in range(8):
        i = g.add(I)
        a, b = g.add_serial_chain([G, E, C])
        g.connect(i, a)
        ends.append(b)
    m0, m1 = g.add(M), g.add(M)
    for k, b in enumerate(ends):
        g.connect(b, m0 if k < 4 else m1)
    o = g.add(O)
    g.connect(m0, o)
    g.connect(m1, o)
    return g


def console_cfg2(seed=2, tracks=64, levels=4, chain=(G, E, C, S, G)) -> Graph:
    """64 tracks i->g->e->c->s->g nested into 4 subgroup levels (fan-in U{2..8})."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = Graph()
    heads = []
    for _ in range(tracks):
        i = g.add(I)
        a, b = g.add_serial_chain(list(chain))
        g.connect(i, a)
        heads.append(b)
    return _subgroups(rng, g, heads, levels)


def random_console(rng, budget_lo=16, budget_hi=256, depth_lo=1, depth_hi=4,
                   chain_lo=1, chain_hi=5, kinds=(G, E, C, S, D)) -> Graph:
    """A random console: tracks with random processor chains, nested subgroups.
    Tracks are added until the node budget (drawn U{budget_lo..budget_hi}) would
    be exceeded by the next track plus its share of mix nodes."""
    budget = int(rng.integers(budget_lo, budget_hi + 1))
    depth = int(rng.integers(depth_lo, depth_hi + 1))
    g = Graph()
    heads = []
    while True:
        n_chain = int(rng.integers(chain_lo, chain_hi + 1))
        # reserve roughly one mix node per 2 tracks per level plus the output
        reserve = 1 + depth * (len(heads) + 1) // 2
        if heads and g.n_nodes + 1 + n_chain + reserve > budget:
            break
        chain = [int(kinds[int(rng.integers(0, len(kinds)))]) for _ in range(n_chain)]
        i = g.add(I)
        a, b = g.add_serial_chain(chain)
        g.connect(i, a)
        heads.append(b)
    return _subgroups(rng, g, heads, depth)


def batch_cfg3(seed=3, n_graphs=128, l_lo=2 ** 15, l_hi=2 ** 18):
    """128 random consoles of uneven size and length; returns (graphs, lengths)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    graphs, lengths = [], []
    for _ in range(n_graphs):
        graphs.append(random_console(rng))
        lengths.append(int(rng.integers(l_lo, l_hi + 1)))
    return graphs, lengths


def console_all_types(seed=4, nodes=200) -> Graph:
    """A console of at least ``nodes`` nodes (the first draw with the node budget raised
    one at a time from ``nodes`` until the console reaches that size) whose chains draw
    from every processor type incl. reverb.  seed 4, 200 nodes: 201 nodes."""
    for budget in range(nodes, 4 * nodes):
        rng = np.random.Generator(np.random.PCG64(seed))
        g = random_console(rng, budget_lo=budget, budget_hi=budget, depth_lo=3, depth_hi=3,
                           chain_lo=2, chain_hi=6, kinds=(G, E, C, S, D, R))
        if g.n_nodes >= nodes:
            return g
    return g

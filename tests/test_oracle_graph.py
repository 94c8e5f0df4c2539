"""Pins for the oracle's graph side: schedule conditions, schedule-length order,
brute force, relabelling invariance and the index maps (Sec. 2, Algorithm 1)."""
import itertools
import json
import os

import numpy as np
import pytest

import synth
from oracle import graph as og
from tests.helpers import random_dag, permute_graph

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def letters(s):
    return "".join(synth.TYPE_LETTERS[t] for t in s)


def brute_force_shortest(types, edges):
    """All type strings by depth-first enumeration (no search heuristics)."""
    n = len(types)
    preds, _ = og.preds_succs(n, edges)
    non_out = frozenset(v for v in range(n) if types[v] != og.O_TYPE)
    ptypes = sorted(set(t for t in types if t not in (0, 1)))
    best = [None]

    def ready(sched, t):
        return frozenset(v for v in range(n) if types[v] == t and v not in sched
                         and all(p in sched for p in preds[v]))

    def dfs(sched, string):
        if sched >= non_out:
            cand = (0,) + string + (1,)
            if best[0] is None or (len(cand), cand) < (len(best[0]), best[0]):
                best[0] = cand
            return
        if best[0] is not None and len(string) + 2 >= len(best[0]):
            return
        for t in ptypes:
            r = ready(sched, t)
            if r:
                dfs(sched | r, string + (t,))

    dfs(frozenset(v for v in range(n) if types[v] == 0), ())
    return best[0]


def test_cfg1_schedule_is_chain_depth():
    g = synth.console_cfg1()
    for m in ("greedy", "beam", "optimal", "one_by_one"):
        s, steps = og.schedule(g.types, g.edges, m)
        og.check_schedule(g.types, g.edges, steps)
        if m != "one_by_one":
            assert letters(s) == "igecmo"
    assert len(og.schedule(g.types, g.edges, "one_by_one")[0]) == 35 - 8 - 1 + 2


@pytest.mark.parametrize("seed", range(40))
def test_schedule_conditions_and_order(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    g = random_dag(rng, n_inputs=int(rng.integers(1, 4)), n_mid=int(rng.integers(2, 9)),
                   n_outputs=int(rng.integers(1, 3)))
    lens = {}
    for m in ("optimal", "beam", "greedy", "one_by_one"):
        s, steps = og.schedule(g.types, g.edges, m, 32)
        og.check_schedule(g.types, g.edges, steps)
        lens[m] = len(s)
    assert lens["optimal"] <= lens["beam"] <= lens["greedy"] <= lens["one_by_one"]
    # Beam(1) is greedy
    assert og.schedule(g.types, g.edges, "beam", 1)[0] == og.schedule(g.types, g.edges, "greedy")[0]
    # the optimal string is the smallest shortest one that brute force finds
    bf = brute_force_shortest(g.types, g.edges)
    assert og.schedule(g.types, g.edges, "optimal")[0] == bf


def longest_processing_path(types, edges):
    n = len(types)
    preds, _ = og.preds_succs(n, edges)
    depth = [0] * n
    order = og.schedule(types, edges, "one_by_one")[1]
    for st in order:
        for v in st:
            if types[v] == 0:
                continue
            depth[v] = 1 + max(depth[p] for p in preds[v])
    return max(depth)


@pytest.mark.parametrize("seed", range(20))
def test_optimal_at_least_longest_path(seed):
    rng = np.random.Generator(np.random.PCG64(100 + seed))
    g = random_dag(rng, n_mid=int(rng.integers(2, 9)))
    s, _ = og.schedule(g.types, g.edges, "optimal")
    assert len(s) - 1 >= longest_processing_path(g.types, g.edges)


@pytest.mark.parametrize("seed", range(10))
def test_relabelling_invariance_of_type_string(seed):
    rng = np.random.Generator(np.random.PCG64(200 + seed))
    g = random_dag(rng, n_mid=9)
    perm = list(rng.permutation(g.n_nodes))
    h = permute_graph(g, perm)
    for m in ("greedy", "beam", "optimal"):
        assert og.schedule(g.types, g.edges, m)[0] == og.schedule(h.types, h.edges, m)[0]


@pytest.mark.parametrize("seed", range(10))
def test_index_maps_consistent(seed):
    rng = np.random.Generator(np.random.PCG64(300 + seed))
    g = random_dag(rng, n_mid=10, n_outputs=2)
    s, steps = og.schedule(g.types, g.edges, "beam")
    mp = og.index_maps(g.types, g.edges, steps)
    sig = mp["sigma"]
    assert sorted(sig) == list(range(g.n_nodes))
    # each step is the contiguous range [step_ptr[n], step_ptr[n+1])
    for k, st in enumerate(steps):
        assert sorted(sig[v] for v in st) == list(range(mp["step_ptr"][k], mp["step_ptr"][k + 1]))
        for v in range(mp["step_ptr"][k], mp["step_ptr"][k + 1]):
            assert mp["types"][v] == s[k]
    # CSR (I^G / I^A) and its transpose reproduce the edge multiset
    e_new = sorted((sig[a], sig[b]) for a, b in g.edges)
    from_csr = sorted((mp["csr_src"][e], d) for d in range(g.n_nodes)
                      for e in range(mp["csr_ptr"][d], mp["csr_ptr"][d + 1]))
    from_t = sorted((s_, mp["tcsr_dst"][e]) for s_ in range(g.n_nodes)
                    for e in range(mp["tcsr_ptr"][s_], mp["tcsr_ptr"][s_ + 1]))
    assert e_new == from_csr == from_t
    # I^P: the l-th type-t node in original order owns row l of P[t]
    inv = {sig[v]: v for v in range(g.n_nodes)}
    for vn in range(g.n_nodes):
        vo = inv[vn]
        assert mp["param_row"][vn] == sum(1 for u in range(vo) if g.types[u] == g.types[vo])


def test_validation_errors():
    I, O, M, G = 0, 1, 2, 3
    with pytest.raises(og.GraphError) as e:
        og.validate([I, G, G, O], [(0, 1), (1, 2), (2, 1), (2, 3)])
    assert e.value.code == "ECYCLE"
    with pytest.raises(og.GraphError):
        og.validate([I, G, O], [(1, 0), (0, 1), (1, 2)])     # input with an in-edge
    with pytest.raises(og.GraphError):
        og.validate([I, G, G, O], [(0, 1), (1, 3)])           # dangling processor
    with pytest.raises(og.GraphError):
        og.validate([I, O, G], [(0, 1), (1, 2)])              # output with an out-edge
    with pytest.raises(og.GraphError):
        og.validate([I, G], [(0, 1)])                         # no output
    with pytest.raises(og.GraphError) as e:
        og.validate([I, 42, O], [(0, 1), (1, 2)])
    assert e.value.code == "ETYPE"


def test_union_is_disconnected_graph():
    rng = np.random.Generator(np.random.PCG64(7))
    gs = [random_dag(rng, n_mid=5) for _ in range(3)]
    types, edges, offs = og.union(gs)
    s, steps = og.schedule(types, edges, "beam")
    og.check_schedule(types, edges, steps)
    # graph-level batching never needs more steps than the longest single schedule
    # would if the types lined up, and never fewer than any one graph's optimum
    assert len(s) >= max(len(og.schedule(g.types, g.edges, "optimal")[0]) for g in gs)


def test_paper_presets_param_sizes():
    """Parameter counts printed in Sec. 3 follow from the processor designs."""
    with open(os.path.join(GOLD, "paper_param_sizes.json")) as f:
        gold = json.load(f)
    from oracle import processors as op
    N = gold["eq_taps"]
    assert (N + 1) // 2 == gold["eq_params"]
    assert op.eq_band_matrix(N).shape[0] == gold["eq_params"]
    assert 2 * 2 * gold["reverb_mags"] == gold["reverb_params"]
    assert gold["delay_delays"] * (2 + gold["delay_mags"]) == gold["delay_params"]
    assert (gold["delay_fir_taps"] + 1) // 2 == gold["delay_mags"]
    assert gold["gain_params"] == synth.PARAM_COLS[synth.G]
    assert gold["imager_params"] == synth.PARAM_COLS[synth.S]
    assert gold["compressor_params"] == synth.PARAM_COLS[synth.C]

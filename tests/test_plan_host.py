"""Host side of the C-ABI library, no GPU: it loads, exports every symbol declared in
include/grafx.h, and its schedules and index maps (Algorithm 1's ScheduleBatchedProcessing
and GetReadWriteIndex) equal the oracle's bit for bit."""
import os
import re

import numpy as np
import pytest

import synth
from oracle import graph as og
from tests.helpers import random_dag

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gx():
    from paper_2408_03204_b300 import build
    build.build()
    import paper_2408_03204_b300 as gx
    gx.lib()
    return gx


def test_exports_every_declared_symbol(gx):
    header = open(os.path.join(ROOT, "include", "grafx.h")).read()
    header = re.sub(r"/\*.*?\*/", "", header, flags=re.S)
    declared = set(re.findall(r"\b(grafx_[a-z0-9_]+)\s*\(", header))
    assert len(declared) >= 20
    lib = gx.lib()
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(gx.SIGNATURES), declared ^ set(gx.SIGNATURES)


def _to_gx(gx, g):
    return gx.Graph.from_lists(g.types, g.edges)


def _compare(gx, graphs, method, width=32, lengths=None):
    lengths = lengths or [1024] * len(graphs)
    plan = gx.Plan([_to_gx(gx, g) for g in graphs], lengths, schedule=method, beam_width=width, eq_taps=31)
    got = plan.export()
    types, edges, _ = og.union(graphs)
    s, steps = og.schedule(types, edges, method, width)
    want = og.index_maps(types, edges, steps)
    assert got["type_string"] == list(s)
    for k in ("step_ptr", "sigma", "csr_ptr", "csr_src", "tcsr_ptr", "tcsr_dst", "param_row"):
        assert got[k] == list(want[k]), k
    return plan


@pytest.mark.parametrize("method", ["beam", "greedy", "optimal", "one_by_one"])
@pytest.mark.parametrize("seed", range(12))
def test_schedule_and_maps_bit_exact_random(gx, method, seed):
    rng = np.random.Generator(np.random.PCG64(1000 + seed))
    g = random_dag(rng, n_inputs=int(rng.integers(1, 4)), n_mid=int(rng.integers(2, 10)),
                   n_outputs=int(rng.integers(1, 3)))
    _compare(gx, [g], method)


@pytest.mark.parametrize("width", [1, 2, 4, 32])
def test_beam_widths_bit_exact(gx, width):
    rng = np.random.Generator(np.random.PCG64(77))
    for _ in range(5):
        _compare(gx, [random_dag(rng, n_mid=14)], "beam", width)


def test_consoles_bit_exact(gx):
    p = _compare(gx, [synth.console_cfg1()], "beam")
    assert p.info.n_steps == 5
    _compare(gx, [synth.console_cfg2()], "beam")
    _compare(gx, [synth.console_cfg2()], "greedy")


def test_batched_union_bit_exact(gx):
    rng = np.random.Generator(np.random.PCG64(3))
    graphs = [synth.random_console(rng, budget_lo=16, budget_hi=64, kinds=(3, 4, 5, 6))
              for _ in range(12)]
    lengths = [int(rng.integers(3000, 9000)) for _ in graphs]
    p = _compare(gx, graphs, "beam", lengths=lengths)
    assert p.info.n_graphs == 12
    assert p.info.src_elems == sum(g.count(0) * 2 * ((L + 3) // 4 * 4) for g, L in zip(graphs, lengths))


def test_error_codes_match_oracle(gx):
    I, O, M, G = 0, 1, 2, 3
    cases = [([I, G, G, O], [(0, 1), (1, 2), (2, 1), (2, 3)], "ECYCLE"),
             ([I, G, O], [(1, 0), (0, 1), (1, 2)], "EINVAL"),
             ([I, G, G, O], [(0, 1), (1, 3)], "EINVAL"),
             ([I, O, G], [(0, 1), (1, 2)], "EINVAL"),
             ([I, G], [(0, 1)], "EINVAL")]
    for types, edges, code in cases:
        with pytest.raises(og.GraphError) as e:
            og.validate(types, edges)
        assert e.value.code == code
        with pytest.raises(gx.GrafxError) as e2:
            gx.Plan([gx.Graph.from_lists(types, edges)], [4096])
        assert e2.value.name == code
    g = gx.Graph()
    with pytest.raises(gx.GrafxError) as e3:
        g.add(42)
    assert e3.value.name == "ETYPE"


def test_bad_options_rejected(gx):
    g = _to_gx(gx, synth.console_cfg1())
    # eq_fft=1024 with 601 taps leaves S = 424 outputs per block < 2H = 600
    for kw in (dict(eq_taps=1024), dict(eq_taps=1), dict(eq_fft=3000), dict(comp_chunk=777),
               dict(eq_taps=601, eq_fft=1024)):
        with pytest.raises(gx.GrafxError):
            gx.Plan([g], [4096], **kw)
    with pytest.raises(gx.GrafxError):
        gx.Plan([g], [0])


def test_paper_layout_widths_and_bad_layouts(gx):
    """The paper's processor settings (Sec. 3) as plan options: parameter widths from the
    plan match the paper's sizes; unknown layouts and sample rates the slot delay cannot
    cover are rejected."""
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_param_sizes.json")))
    g = gx.Graph.from_lists([0, 5, 7, 8, 3, 4, 6, 9, 1], [(0, 1), (1, 2), (2, 3), (3, 4), (4, 5), (5, 6),
                                                         (6, 7), (7, 8)])
    p = gx.Plan([g], [8192], preset="paper")
    assert p.param_cols[5] == gold["eq_params"] and p.param_cols[7] == gold["delay_params"]
    assert p.param_cols[8] == gold["reverb_params"] and p.param_cols[3] == gold["gain_params"]
    assert p.param_cols[4] == gold["imager_params"] and p.param_cols[6] == gold["compressor_params"]
    c = gx.Plan([g], [8192])
    assert c.param_cols == {3: 2, 4: 1, 5: 8, 6: 4, 7: 176, 8: 50, 9: 4, 12: 4, 13: 5}
    # one setting of the preset overridden: band EQ on the paper's other layouts
    m = gx.Plan([g], [8192], preset="paper", eq_params="bands")
    assert m.param_cols[5] == 8 and m.param_cols[7] == 880
    # EQ log-magnitudes follow eq_taps
    assert gx.Plan([g], [8192], eq_params="logmag", eq_taps=255).param_cols[5] == 128
    o = gx.PlanOpts()
    gx.lib().grafx_plan_opts_default(gx.ctypes.byref(o))
    for field, bad in (("eq_params", 2), ("delay_layout", 5), ("reverb_layout", -1)):
        o2 = gx.PlanOpts.from_buffer_copy(o)
        setattr(o2, field, bad)
        h = gx._P()
        hs = (gx._P * 1)(g._h)
        ls = (gx.ctypes.c_int64 * 1)(8192)
        assert gx.lib().grafx_plan_create(hs, 1, ls, gx.ctypes.byref(o2), gx.ctypes.byref(h)) == 1
    with pytest.raises(gx.GrafxError):
        gx.Plan([g], [8192], preset="paper", sample_rate=96000)
    gx.Plan([g], [8192], preset="paper", sample_rate=48000)


def test_source_batch_rows(gx):
    """Source-level batch (Sec. 2 "Batched processing"): B copies of the graph share the
    parameter rows of one pass (I^P of every copy equals copy 0's); sources and outputs
    grow by B; a partial backward range is refused."""
    g = synth.console_cfg1()
    h = _to_gx(gx, g)
    one = gx.Plan([h], [4096])
    three = gx.Plan([h], [4096], source_batch=3)
    assert three.info.source_batch == 3 and one.info.source_batch == 1
    assert list(three.info.n_type_rows) == list(one.info.n_type_rows)
    assert three.info.src_elems == 3 * one.info.src_elems and three.info.out_elems == 3 * one.info.out_elems
    assert three.info.n_nodes == 3 * one.info.n_nodes and three.info.node_samples == 3 * one.info.node_samples
    e1, e3 = one.export(), three.export()
    assert e3["type_string"] == e1["type_string"]          # the copies run in the same steps
    n = one.info.n_nodes
    # new id of copy b's node v is sigma3[b n + v]; its parameter row is copy 0's
    for b in range(3):
        for v in range(n):
            assert e3["param_row"][e3["sigma"][b * n + v]] == e1["param_row"][e1["sigma"][v]]
    with pytest.raises(gx.GrafxError):
        gx.Plan([h], [4096], source_batch=-2)


def test_type_ports_and_port_checks(gx):
    """Eq. 1a: the port counts of every type; an edge must leave an existing output and
    enter an existing input (checked when connecting and when planning)."""
    want = {0: (0, 1), 1: (1, 1), 10: (1, 2), 11: (2, 1), 12: (2, 1)}
    for t in range(gx.N_TYPES):
        assert gx.type_ports(t) == want.get(t, (1, 1))
    with pytest.raises(gx.GrafxError):
        gx.type_ports(14)
    g = gx.Graph()
    i, sp, mg, o = g.add(0), g.add(10), g.add(11), g.add(1)
    g.connect(i, sp)
    g.connect(sp, mg, 0, 0)
    g.connect(sp, mg, 1, 1)
    g.connect(mg, o)
    for bad in ((sp, mg, 2, 0), (sp, mg, 0, 2), (i, sp, 1, 0), (mg, o, 0, 1)):
        with pytest.raises(gx.GrafxError) as e:
            g.connect(*bad)
        assert e.value.name == "EINVAL"
    p = gx.Plan([g], [4096])
    assert p.info.n_steps >= 3


def test_optimal_size_limit(gx):
    rng = np.random.Generator(np.random.PCG64(5))
    g = random_dag(rng, n_mid=40)
    with pytest.raises(gx.GrafxError):
        gx.Plan([_to_gx(gx, g)], [4096], schedule="optimal")


def test_workspace_requires_binding(gx):
    p = gx.Plan([_to_gx(gx, synth.console_cfg1())], [4096])
    with pytest.raises(gx.GrafxError) as e:
        p.render_raw(None, None, None)
    assert e.value.name == "EINVAL"


def test_delay_and_reverb_length_limit(gx):
    I, O, D, R = 0, 1, 7, 8
    for t in (D, R):
        ok = gx.Graph.from_lists([I, t, O], [(0, 1), (1, 2)])
        gx.Plan([ok], [1 << 19])
        with pytest.raises(gx.GrafxError) as e:
            gx.Plan([ok], [(1 << 19) + 1])
        assert e.value.name == "ESHAPE"


def test_checkpointing_shrinks_the_workspace(gx):
    g = _to_gx(gx, synth.console_cfg2())
    row = 2 * (1 << 17) * 4
    base = gx.Plan([g], [1 << 17]).info.ws_bytes
    size = {k: gx.Plan([g], [1 << 17], checkpoint_steps=k).info.ws_bytes for k in (1, 2, 3, 100)}
    # a consumer always runs in a later step: one-step segments keep every row, and one
    # segment spanning the schedule holds every row in its scratch region (the plan
    # without checkpointing fuses the imager and last gain steps, which keeps the
    # imagers' adjoint rows one step longer: at least as large)
    assert size[1] == size[100] and size[1] <= base
    # cfg2's chains (g e c s g) cut into 2- or 3-step segments recycle one row per track
    # and segment boundary crossed inside a segment: at least 64 rows fewer
    assert size[2] < base - 64 * row and size[3] < base - 64 * row
    with pytest.raises(gx.GrafxError):
        gx.Plan([g], [4096], checkpoint_steps=-1)


def test_adjoint_rows_are_recycled(gx):
    """Adjoint rows live from their node's backward step to their producers' steps; the
    chains of cfg2 need far fewer rows than one per internal node."""
    cfg2 = synth.console_cfg2()
    g = _to_gx(gx, cfg2)
    L = 1 << 17
    row = 2 * L * 4
    internal = sum(1 for t in cfg2.types if t not in (synth.I, synth.O))
    info = gx.Plan([g], [L]).info
    # the EQ's per-block input spectra (kept by the forward for the backward): M bins of
    # 8 bytes per overlap-save block, S = M - 2H outputs per block (1023 taps)
    M, H = info.eq_fft, 511
    Hal, S = (H + 3) & ~3, (info.eq_fft - 2 * H) & ~3
    spectra = cfg2.types.count(synth.E) * ((L + Hal - H + S - 1) // S) * M * 8
    # workspace = U (one row per internal node) + A + spectra + small tables; A < internal / 2 rows
    assert info.ws_bytes < (internal + internal / 2) * row + spectra + 64 * 2 ** 20


def test_schedule_benchmark_consoles_step_counts(gx):
    """The schedule-method benchmark's consoles: the exact search is never beaten, and
    type scheduling needs far fewer steps than one node per step on the larger ones."""
    from paper_2408_03204_b300 import schedules as S
    gs = S.consoles(8, seed=5)
    for g in gs:
        n_proc = sum(1 for t in g.types if t not in (synth.I, synth.O))
        steps = {m: gx.Plan([_to_gx(gx, g)], [4096], schedule=m).info.n_steps
                 for m in S.METHODS if m != "optimal" or n_proc <= S.OPTIMAL_MAX_PROC}
        if "optimal" in steps:
            assert steps["optimal"] <= min(steps.values())
        assert steps["one_by_one"] == n_proc + 1 or steps["one_by_one"] >= steps["beam"]
    big = gs[-1]
    nb = gx.Plan([_to_gx(gx, big)], [4096], schedule="beam").info.n_steps
    no = gx.Plan([_to_gx(gx, big)], [4096], schedule="one_by_one").info.n_steps
    assert no >= 2 * nb


def test_fused_elementwise_step_pairs(gx):
    """The nested console's first gain step feeds its EQ step, its imager step its last
    gain step and its master mix its output node for node: three fused pairs; none with
    checkpointing; none when an imager feeds two gains."""
    cfg2 = _to_gx(gx, synth.console_cfg2())
    assert gx.Plan([cfg2], [4096]).info.fused_pairs == 3
    assert gx.Plan([cfg2], [4096], checkpoint_steps=2).info.fused_pairs == 0
    g = synth.Graph()
    i, s = g.add(synth.I), g.add(synth.S)
    g1, g2, o = g.add(synth.G), g.add(synth.G), g.add(synth.O)
    g.connect(i, s)
    g.connect(s, g1)
    g.connect(s, g2)
    g.connect(g1, o)
    g.connect(g2, o)
    assert gx.Plan([_to_gx(gx, g)], [4096]).info.fused_pairs == 0
    h = synth.Graph()
    i, s, g1, o = h.add(synth.I), h.add(synth.S), h.add(synth.G), h.add(synth.O)
    h.connect(i, s)
    h.connect(s, g1)
    h.connect(g1, o)
    assert gx.Plan([_to_gx(gx, h)], [4096]).info.fused_pairs == 1   # g -> o is not a pair
    q = synth.Graph()
    i, g1, e, o = q.add(synth.I), q.add(synth.G), q.add(synth.E), q.add(synth.O)
    q.connect(i, g1)
    q.connect(g1, e)
    q.connect(e, o)
    assert gx.Plan([_to_gx(gx, q)], [4096]).info.fused_pairs == 1


def test_compressor_items_chunk_major(gx):
    """The compressor's one-pass kernels take their chunks by ticket in item order and
    find a node's other chunks through their chunk id (forward) or partial slot
    (backward): the items are chunk-major (the c-th chunk of every node before any
    node's (c+1)-th; the backward from each node's end), every chunk of every node once,
    ids and slots contiguous per node in node order, and the step's first item is its
    first node's first chunk (forward) or last chunk (backward)."""
    G, E, C = synth.G, synth.E, synth.C
    rng = np.random.Generator(np.random.PCG64(5))
    graphs = [synth.random_console(rng, budget_lo=16, budget_hi=40, kinds=(G, E, C)) for _ in range(4)]
    lengths = [int(rng.integers(3000, 20000)) for _ in graphs]
    plan = gx.Plan([_to_gx(gx, g) for g in graphs], lengths, comp_chunk=1024)
    ex = plan.export()
    new_len = {}
    base = 0
    for g, L in zip(graphs, lengths):
        for v in range(g.n_nodes):
            new_len[ex["sigma"][base + v]] = L
        base += g.n_nodes
    steps = [k for k in range(1, len(ex["type_string"])) if ex["type_string"][k] == C]
    assert steps
    for k in steps:
        nodes = list(range(ex["step_ptr"][k], ex["step_ptr"][k + 1]))
        nc = {v: (new_len[v] + 1023) // 1024 for v in nodes}
        fwd = plan.step_items(k)
        bwd = plan.step_items(k, backward=True)
        want_f = [(v, c) for c in range(max(nc.values())) for v in nodes if c < nc[v]]
        want_b = [(v, nc[v] - 1 - r) for r in range(max(nc.values())) for v in nodes if r < nc[v]]
        assert [tuple(x) for x in fwd[:, :2]] == want_f
        assert [tuple(x) for x in bwd[:, :2]] == want_b
        # chunk ids (both directions) and partial slots (backward) contiguous per node
        cid = {(v, c): z for v, c, z, _ in fwd}
        assert all(cid[(v, c)] == z for v, c, z, _ in bwd)
        first_id = {v: cid[(v, 0)] for v in nodes}
        slot = {(v, c): s for v, c, _, s in bwd}
        first_slot = {v: slot[(v, nc[v] - 1)] for v in nodes}
        for i, v in enumerate(nodes):
            assert [cid[(v, c)] for c in range(nc[v])] == list(range(first_id[v], first_id[v] + nc[v]))
            assert [slot[(v, nc[v] - 1 - r)] for r in range(nc[v])] == list(range(first_slot[v], first_slot[v] + nc[v]))
            if i:
                assert first_id[v] == first_id[nodes[i - 1]] + nc[nodes[i - 1]]
                assert first_slot[v] == first_slot[nodes[i - 1]] + nc[nodes[i - 1]]
        assert fwd[0][2] == min(cid.values()) and bwd[0][3] == min(slot.values())


def test_readme_quickstart_plan(gx):
    """The host half of the README's quick start: its graph plans to the schedule
    i g e c m o, its buffers have the documented layouts and its parameter tables the
    widths the example allocates."""
    L = 2 ** 17
    g = gx.Graph()
    tracks = [g.add(gx.T_IN) for _ in range(4)]
    bus, out = g.add(gx.T_MIX), g.add(gx.T_OUT)
    for i in tracks:
        first, last = g.add_serial_chain([gx.T_GAIN, gx.T_EQ, gx.T_COMP])
        g.connect(i, first)
        g.connect(last, bus)
    g.connect(bus, out)
    plan = gx.Plan([g], [L])
    info = plan.info
    assert info.src_elems == 4 * 2 * gx.pitch(L)      # [input][2][pitch(L)]
    assert info.out_elems == 1 * 2 * gx.pitch(L)      # [output][2][pitch(L)]
    assert [info.n_type_rows[t] for t in (gx.T_GAIN, gx.T_EQ, gx.T_COMP, gx.T_MIX)] == [4, 4, 4, 1]
    assert (plan.param_cols[gx.T_GAIN], plan.param_cols[gx.T_EQ], plan.param_cols[gx.T_COMP]) == (2, 8, 4)
    assert "".join(synth.TYPE_LETTERS[t] for t in plan.export()["type_string"]) == "igecmo"

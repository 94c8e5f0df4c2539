"""GPU parity of multi-port nodes (Sec. 2 Definitions, Eq. 1a/1b with M inputs, N outputs
and typed edges) against the FP64 oracle: split, merge and the sidechain compressor in
random graphs, batched with ragged lengths, forward and backward, with and without
signal checkpointing, at every compressor chunk size."""
import numpy as np
import pytest

import synth
from oracle import render as orr
from tests.gpu_common import DeviceRun, assert_grad_close, assert_out_close, flat_sources, per_graph_params, split_rows, union_params
from tests.helpers import random_mimo_dag

pytestmark = pytest.mark.gpu

HP = dict(eq_taps=63)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")


def check(graphs, lengths, seed, **plan_kw):
    src_flat, src_per = flat_sources(graphs, lengths, [seed + k for k in range(len(graphs))])
    P = union_params(graphs, seed)
    run = DeviceRun(graphs, lengths, P, src_flat, eq_taps=63, **plan_kw)
    out = run.render().cpu().numpy()
    Pg = per_graph_params(graphs, P)
    rng = np.random.Generator(np.random.PCG64(seed))
    Ws, wants = [], []
    for g, L, src, p, got in zip(graphs, lengths, src_per, Pg, split_rows(out, graphs, lengths)):
        want = orr.outputs_of(g.types, orr.render_one_by_one(g.types, g.edges, src[:, :, :L], p, HP, ports=g.ports))
        assert_out_close(got, want)
        Pd = (L + 3) // 4 * 4
        W = np.zeros((g.count(synth.O), 2, Pd), np.float32)
        W[:, :, :L] = rng.standard_normal((g.count(synth.O), 2, L)).astype(np.float32)
        Ws.append(W)
    dP, dS = run.backprop(np.concatenate([w.reshape(-1) for w in Ws]))
    off, cnt = 0, {}
    for g, L, src, p, W in zip(graphs, lengths, src_per, Pg, Ws):
        wP, wS, wC = orr.backward(g.types, g.edges, src[:, :, :L], p, W[:, :, :L], HP, cond=True, ports=g.ports)
        Pd = (L + 3) // 4 * 4
        K = g.count(synth.I)
        assert_grad_close(dS[off:off + K * 2 * Pd].reshape(K, 2, Pd)[:, :, :L], wS, what="sources")
        off += K * 2 * Pd
        for t in wP:
            n = g.count(t)
            a = cnt.get(t, 0)
            assert_grad_close(dP[t][a:a + n], wP[t], what=f"type {t}", cond=wC[t])
            cnt[t] = a + n
    return run


def test_mid_side_round_trip_is_exact_on_the_gpu():
    g = synth.Graph()
    i = g.add(synth.I)
    sp = g.add(synth.P)
    mg = g.add(synth.J)
    o = g.add(synth.O)
    g.connect(i, sp)
    g.connect(sp, mg, 0, 0)
    g.connect(sp, mg, 1, 1)
    g.connect(mg, o)
    L = 10007
    src_flat, src_per = flat_sources([g], [L], [3])
    run = DeviceRun([g], [L], {}, src_flat)
    out = run.render().cpu().numpy()
    got = split_rows(out, [g], [L])[0]
    np.testing.assert_allclose(got[0], src_per[0][0, :, :L], atol=1e-6)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_mimo_graphs(seed):
    rng = np.random.Generator(np.random.PCG64(100 + seed))
    graphs = [random_mimo_dag(rng, 3, 12, 2) for _ in range(3)]
    lengths = [int(rng.integers(3000, 11000)) for _ in graphs]
    check(graphs, lengths, 500 + seed)


def test_mimo_with_checkpointing():
    rng = np.random.Generator(np.random.PCG64(7))
    graphs = [random_mimo_dag(rng, 3, 16, 1)]
    check(graphs, [9001], 77, checkpoint_steps=2)


@pytest.mark.parametrize("chunk", [1024, 4096])
def test_sidechain_chunk_sizes(chunk):
    rng = np.random.Generator(np.random.PCG64(chunk + 1))
    kinds = (synth.K, synth.G, synth.P, synth.J)
    graphs = [random_mimo_dag(rng, 2, 8, 1, kinds=kinds)]
    check(graphs, [3 * chunk + 77], chunk, comp_chunk=chunk)

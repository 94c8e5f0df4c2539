"""Degenerate signal lengths through every processor type on the GPU, against the FP64
oracle: signals of 1 to 255 samples (shorter than one tile, FFT block, compressor chunk,
delay or reverb block), forward and backward, one graph per length and all lengths
batched ragged in one plan."""
import numpy as np
import pytest

import synth
from oracle import render as orr
from tests.gpu_common import assert_grad_close
from tests.helpers import random_dag
from tests.test_gpu_parity import run_case

pytestmark = pytest.mark.gpu

KINDS = (synth.M, synth.G, synth.S, synth.E, synth.C, synth.N, synth.D, synth.R, synth.A)


def _graph(seed):
    """A random DAG over KINDS plus one chain through every processor type, multi-port
    ones included: i -> g -> s -> e -> c -> n -> d -> r -> a -> split -> (gain, gain) ->
    merge -> sidechain (keyed by a second input) -> o."""
    rng = np.random.Generator(np.random.PCG64(seed))
    g = random_dag(rng, n_inputs=2, n_mid=8, n_outputs=1, kinds=KINDS)
    prev = g.add(synth.I)
    for t in KINDS[1:]:
        v = g.add(t)
        g.connect(prev, v)
        prev = v
    sp, gm, gs, mg = g.add(synth.P), g.add(synth.G), g.add(synth.G), g.add(synth.J)
    key, sc, o = g.add(synth.I), g.add(synth.K), g.add(synth.O)
    g.connect(prev, sp)
    g.connect(sp, gm, 0, 0)
    g.connect(sp, gs, 1, 0)
    g.connect(gm, mg, 0, 0)
    g.connect(gs, mg, 0, 1)
    g.connect(mg, sc, 0, 0)
    g.connect(key, sc, 0, 1)
    g.connect(sc, o)
    return g


def _backward_check(run, graphs, lengths, P, src_per, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    Ws, flat = [], []
    for g, L in zip(graphs, lengths):
        Pd = (L + 3) // 4 * 4
        W = np.zeros((g.count(synth.O), 2, Pd), np.float32)
        W[:, :, :L] = rng.standard_normal((g.count(synth.O), 2, L)).astype(np.float32)
        Ws.append(W)
        flat.append(W.reshape(-1))
    dP, dS = run.backprop(np.concatenate(flat))
    off, rows = 0, {t: 0 for t in P}
    hp = dict(eq_taps=63, reverb_noise=synth.reverb_noise().astype(np.float64))
    for g, L, src, W in zip(graphs, lengths, src_per, Ws):
        p = {}
        for t in P:
            n = g.count(t)
            if n:
                p[t] = P[t][rows[t]:rows[t] + n]
        wP, wS, wC = orr.backward(g.types, g.edges, src[:, :, :L], p, W[:, :, :L], hp, cond=True, ports=g.ports)
        for t in p:
            assert_grad_close(dP[t][rows[t]:rows[t] + g.count(t)], wP[t], what=f"L={L} type {t}", cond=wC[t])
            rows[t] += g.count(t)
        Pd = (L + 3) // 4 * 4
        n = g.count(synth.I) * 2 * Pd
        assert_grad_close(dS[off:off + n].reshape(-1, 2, Pd)[:, :, :L], wS, what=f"L={L} sources")
        off += n


@pytest.mark.parametrize("L", [1, 2, 3, 5, 17, 255])
def test_tiny_lengths_every_processor(L):
    g = _graph(900 + L)
    run, P, src_per, _ = run_case([g], [L], seed=910 + L)
    _backward_check(run, [g], [L], P, src_per, 920 + L)


def test_tiny_and_long_lengths_batched_ragged():
    lengths = [1, 4099, 3, 255]
    graphs = [_graph(950 + k) for k in range(len(lengths))]
    run, P, src_per, _ = run_case(graphs, lengths, seed=960)
    _backward_check(run, graphs, lengths, P, src_per, 970)

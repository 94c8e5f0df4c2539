"""GPU parity of the compressor with attack/release ballistics (Sec. 3, Eq. 8 with
separate attack and release coefficients; the sample-serial envelope) against the FP64
oracle: single nodes across several 512-sample blocks with ragged tails, nodes sharing a
step, and random graphs, forward and backward."""
import numpy as np
import pytest

import synth
from tests.test_gpu_parity import run_case, single_node_graph
from tests.gpu_common import assert_grad_close
from oracle import render as orr
from tests.helpers import random_dag

pytestmark = pytest.mark.gpu

A = synth.A


def backward_check(run, g, L, P, src, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    Pd = (L + 3) // 4 * 4
    n_out = g.count(synth.O)
    W = np.zeros((n_out, 2, Pd), np.float32)
    W[:, :, :L] = rng.standard_normal((n_out, 2, L)).astype(np.float32)
    dP, dS = run.backprop(W.reshape(-1))
    wP, wS, wC = orr.backward(g.types, g.edges, src[:, :, :L], P, W[:, :, :L], dict(eq_taps=63), cond=True)
    for t in P:
        assert_grad_close(dP[t], wP[t], what=f"type {t}", cond=wC[t])
    assert_grad_close(dS.reshape(-1, 2, Pd)[:, :, :L], wS, what="sources")


@pytest.mark.parametrize("L", [5003, 2 ** 15 + 77])
def test_ballistic_single_node(L):
    g = single_node_graph(A, fan_in=2)
    run, P, src_per, _ = run_case([g], [L], seed=L)
    backward_check(run, g, L, P, src_per[0], L + 1)


def test_ballistic_nodes_sharing_steps_and_random_graphs():
    rng = np.random.Generator(np.random.PCG64(13))
    for k in range(3):
        g = random_dag(rng, n_inputs=2, n_mid=8, n_outputs=1, kinds=(A, synth.G, synth.E, synth.C, synth.M))
        L = int(rng.integers(3000, 9000))
        run, P, src_per, _ = run_case([g], [L], seed=700 + k)
        backward_check(run, g, L, P, src_per[0], 800 + k)


def test_ballistic_coefficient_orders_and_short_signals():
    """A slower attack than release (the envelope takes the smaller candidate step), equal
    coefficients (the one-pole filter) and the usual order, on signals of 3 samples (one
    partial block) and 1029 samples (two blocks and a ragged tail)."""
    from tests.gpu_common import DeviceRun, flat_sources, split_rows

    def bank_graph(n):
        g = synth.Graph()
        for _ in range(n):
            i, v, o = g.add(synth.I), g.add(A), g.add(synth.O)
            g.connect(i, v)
            g.connect(v, o)
        return g
    graphs = [bank_graph(3), bank_graph(3)]
    lengths = [3, 1029]
    src_flat, src_per = flat_sources(graphs, lengths, [41, 42])
    T, W, R = np.log(10 ** (-20 / 10)), 3.0 * np.log(10) / 10, 4.0
    rows = np.array([[0.7, 0.9995, T, W, R], [0.9995, 0.7, T, W, R], [0.98, 0.98, T, W, R]])
    P = {A: np.concatenate([rows, rows])}
    run = DeviceRun(graphs, lengths, P, src_flat)
    got = split_rows(run.render().cpu().numpy(), graphs, lengths)
    Pd = [(L + 3) // 4 * 4 for L in lengths]
    rng = np.random.Generator(np.random.PCG64(5))
    Wf = [np.zeros((3, 2, p), np.float32) for p in Pd]
    for w, L in zip(Wf, lengths):
        w[:, :, :L] = rng.standard_normal((3, 2, L)).astype(np.float32)
    dP, dS = run.backprop(np.concatenate([w.reshape(-1) for w in Wf]))
    off = 0
    for k, (g, L, src) in enumerate(zip(graphs, lengths, src_per)):
        p = {A: rows}
        want = orr.outputs_of(g.types, orr.render_one_by_one(g.types, g.edges, src[:, :, :L], p, dict(eq_taps=63)))
        np.testing.assert_allclose(got[k], want, atol=1e-5 * max(1.0, np.abs(want).max()), rtol=0)
        wP, wS, wC = orr.backward(g.types, g.edges, src[:, :, :L], p, Wf[k][:, :, :L], dict(eq_taps=63), cond=True)
        assert_grad_close(dP[A][3 * k:3 * k + 3], wP[A], what=f"graph {k}", cond=wC[A])
        n = 3 * 2 * Pd[k]
        assert_grad_close(dS[off:off + n].reshape(3, 2, Pd[k])[:, :, :L], wS, what=f"sources {k}")
        off += n

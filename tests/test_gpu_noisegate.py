"""Noisegate (Eq. 13) on the GPU against the FP64 oracle: one gate node over long
signals crossing the knee at both extremes of alpha, and random graphs that mix
gates with the other processors."""
import numpy as np
import pytest

import synth
from oracle import render as orr
from tests.gpu_common import DeviceRun, assert_grad_close, assert_out_close, flat_sources
from tests.test_gpu_parity import run_case, single_node_graph

pytestmark = pytest.mark.gpu
N = synth.N


@pytest.mark.parametrize("alpha", [0.9, 0.9999])
def test_noisegate_long_signal(alpha):
    g = single_node_graph(N)
    L = 2 ** 17 + 8
    src_flat, src_per = flat_sources([g], [L], [6])
    # threshold near the sources' envelope so that all three regions of the curve occur
    P = {N: np.array([[alpha, np.log(0.004), 0.6908, 3.0]], np.float32)}
    run = DeviceRun([g], [L], P, src_flat)
    got = run.render().cpu().numpy().reshape(1, 2, L)
    want = orr.outputs_of(g.types, orr.render_one_by_one(g.types, g.edges, src_per[0], P))
    assert_out_close(got, want)
    W = np.random.Generator(np.random.PCG64(4)).standard_normal((1, 2, L)).astype(np.float32)
    dP, dS = run.backprop(W.reshape(-1))
    wP, wS = orr.backward(g.types, g.edges, src_per[0], P, W)
    assert_grad_close(dP[N], wP[N], what=f"gate alpha={alpha}")
    assert_grad_close(dS.reshape(-1, 2, L), wS, what="sources")


def test_noisegate_ratio_one_passes_through():
    g = single_node_graph(N)
    L = 9001
    src_flat, src_per = flat_sources([g], [L], [8])
    run = DeviceRun([g], [L], {N: np.array([[0.99, -3.0, 0.69, 1.0]], np.float32)}, src_flat)
    got = run.render().cpu().numpy().reshape(1, 2, -1)[:, :, :L]
    assert_out_close(got, src_per[0][:, :, :L])


def test_random_graphs_with_gates():
    from tests.helpers import random_dag
    M, G, E, C, S = synth.M, synth.G, synth.E, synth.C, synth.S
    rng = np.random.Generator(np.random.PCG64(31))
    for k in range(3):
        g = random_dag(rng, n_inputs=3, n_mid=10, n_outputs=2, kinds=(M, G, E, C, N, S))
        L = int(rng.integers(3000, 9000))
        run, P, src_per, out = run_case([g], [L], seed=300 + k)
        Pd = (L + 3) // 4 * 4
        W = np.zeros((2, 2, Pd), np.float32)
        W[:, :, :L] = rng.standard_normal((2, 2, L)).astype(np.float32)
        dP, dS = run.backprop(W.reshape(-1))
        wP, wS, wC = orr.backward(g.types, g.edges, src_per[0][:, :, :L], P, W[:, :, :L], dict(eq_taps=63),
                                  cond=True)
        for t in P:
            assert_grad_close(dP[t], wP[t], what=f"type {t}", cond=wC[t])
        assert_grad_close(dS.reshape(-1, 2, Pd)[:, :, :L], wS, what="sources")


@pytest.mark.parametrize("chunk", [1024, 4096])
def test_compressor_and_gate_other_chunk_sizes(chunk):
    """The 1024- and 4096-sample chunk variants (4 and 16 samples per thread) against the
    oracle, forward and backward."""
    from tests.helpers import random_dag
    rng = np.random.Generator(np.random.PCG64(chunk))
    g = random_dag(rng, n_inputs=2, n_mid=6, n_outputs=1, kinds=(synth.C, N, synth.G))
    L = 3 * chunk + 77
    run, P, src_per, out = run_case([g], [L], seed=chunk, comp_chunk=chunk)
    Pd = (L + 3) // 4 * 4
    W = np.zeros((1, 2, Pd), np.float32)
    W[:, :, :L] = rng.standard_normal((1, 2, L)).astype(np.float32)
    dP, dS = run.backprop(W.reshape(-1))
    wP, wS = orr.backward(g.types, g.edges, src_per[0][:, :, :L], P, W[:, :, :L], dict(eq_taps=63))
    for t in P:
        assert_grad_close(dP[t], wP[t], what=f"type {t} chunk {chunk}")

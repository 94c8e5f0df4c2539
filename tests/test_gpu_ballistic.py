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

"""The largest signals a plan accepts, on the GPU against the FP64 oracle: 2^24 samples
through a chain of gain, EQ, compressor, noisegate and imager, the attack/release
compressor at 2^21 (the oracle's sample loop), and 2^19 samples (the delay and reverb
limit) through a delay and a reverb; forward everywhere, backward through the parameter
gradients and the source adjoint.  Host rejection of the next size up."""
import numpy as np
import pytest

import synth
from oracle import render as orr
from tests.gpu_common import DeviceRun, assert_grad_close, assert_out_close, flat_sources, union_params

pytestmark = pytest.mark.gpu


def _chain(kinds):
    g = synth.Graph()
    prev = g.add(synth.I)
    for t in kinds:
        v = g.add(t)
        g.connect(prev, v)
        prev = v
    o = g.add(synth.O)
    g.connect(prev, o)
    return g


def _check(g, L, seed, eq_taps=63):
    src_flat, src_per = flat_sources([g], [L], [seed])
    P = union_params([g], seed)
    run = DeviceRun([g], [L], P, src_flat, eq_taps=eq_taps)
    got = run.render().cpu().numpy().reshape(-1, 2, (L + 3) // 4 * 4)[:, :, :L]
    hp = dict(eq_taps=eq_taps, reverb_noise=synth.reverb_noise().astype(np.float64))
    src = src_per[0][:, :, :L]
    want = orr.outputs_of(g.types, orr.render_one_by_one(g.types, g.edges, src, P, hp))
    assert_out_close(got, want)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    Pd = (L + 3) // 4 * 4
    W = np.zeros((1, 2, Pd), np.float32)
    W[:, :, :L] = rng.standard_normal((1, 2, L)).astype(np.float32)
    dP, dS = run.backprop(W.reshape(-1))
    del run
    wP, wS, wC = orr.backward(g.types, g.edges, src, P, W[:, :, :L], hp, cond=True)
    for t in P:
        assert_grad_close(dP[t], wP[t], what=f"type {t}", cond=wC[t])
    assert_grad_close(dS.reshape(-1, 2, Pd)[:, :, :L], wS, what="sources")


def test_longest_signal_every_unlimited_processor():
    _check(_chain([synth.G, synth.E, synth.C, synth.N, synth.S]), 2 ** 24, 5)


def test_long_signal_attack_release():
    """The attack/release envelope at 2^21 samples (the oracle's sample loop bounds the
    size; the kernel has no length limit)."""
    _check(_chain([synth.A, synth.G]), 2 ** 21, 7)


def test_longest_signal_with_delay_and_reverb():
    _check(_chain([synth.D, synth.R]), 2 ** 19, 6)


def test_lengths_past_the_limits_are_rejected():
    import paper_2408_03204_b300 as gx
    g = _chain([synth.G])
    with pytest.raises(gx.GrafxError):
        gx.Plan([gx.Graph.from_lists(g.types, g.edges)], [2 ** 24 + 1])
    d = _chain([synth.D])
    with pytest.raises(gx.GrafxError):
        gx.Plan([gx.Graph.from_lists(d.types, d.edges)], [2 ** 19 + 1])

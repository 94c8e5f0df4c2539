"""The full-fit workload's graph at its stated size: a 201-node console whose chains draw
from every processor type, the filtered-noise reverb (1024/256, 12 bands, wet/dry)
included, rendered and differentiated with signal checkpointing every 3 schedule steps
(as the fit runs it), against the FP64 oracle at a ragged 2^15 + 3 samples."""
import numpy as np
import pytest

import synth
from gpu_common import GRAD_TOL, DeviceRun, assert_grad_close, assert_out_close, flat_sources
from oracle import render as orr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2408_03204_b300 import build
    build.build()


def test_all_types_console_with_checkpointing_matches_oracle():
    g = synth.console_all_types()
    assert g.n_nodes >= 200 and g.count(synth.R) > 0 and g.count(synth.D) > 0
    L = 2 ** 15 + 3
    Pd = (L + 3) // 4 * 4
    src_flat, src_per = flat_sources([g], [L], [4])
    P = synth.random_params(g, 104)
    run = DeviceRun([g], [L], P, src_flat, checkpoint_steps=3)
    got = run.render().cpu().numpy().reshape(-1, 2, Pd)
    hp = dict(eq_taps=1023, reverb_noise=synth.reverb_noise().astype(np.float64))
    src = src_per[0][:, :, :L]
    want = orr.outputs_of(g.types, orr.render_one_by_one(g.types, g.edges, src, P, hp))
    assert_out_close(got[:, :, :L], want)
    assert not got[:, :, L:].any()
    W = np.zeros((want.shape[0], 2, Pd), np.float32)
    W[:, :, :L] = np.random.Generator(np.random.PCG64(44)).standard_normal((want.shape[0], 2, L))
    dP, dS = run.backprop(W.reshape(-1))
    wP, wS, wC = orr.backward(g.types, g.edges, src, P, W[:, :, :L], hp, cond=True)
    for t in wP:
        if t == synth.D:
            # the surrogate z-gradient and the FIR log-magnitudes, as the delay tests split them
            q, wq = dP[t].reshape(-1, 2, 4, 22), wP[t].reshape(-1, 2, 4, 22)
            assert_grad_close(q[..., :2], wq[..., :2], GRAD_TOL, what="delay z")
            assert_grad_close(q[..., 2:], wq[..., 2:], GRAD_TOL, what="delay FIR")
        else:
            assert_grad_close(dP[t], wP[t], GRAD_TOL, what=f"type {t}", cond=wC.get(t))
    assert_grad_close(dS.reshape(-1, 2, Pd)[:, :, :L], wS, what="sources")

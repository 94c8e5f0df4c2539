"""The allocation-free compressor call, for callers that must not allocate device memory
(real-time audio callbacks and plugin hosts, where an allocation can stall on a
device-wide synchronisation, and frameworks that own all device memory through their
own pool).  Its output must match the compressor of the ordinary render path on the
same input, on two calls in a row (the second call reuses the library's fixed scratch,
which the first call left dirty), with every padding sample up to the row's pitch zeroed
and no timeout reported in the caller's status word.

This file is named to be collected last, so a run that stops at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest

import synth
from tests.gpu_common import OUT_TOL, DeviceRun, assert_out_close, flat_sources

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2408_03204_b300 import build
    build.build()


def _noalloc_vs_render(L, pitch, seed, status_init=0):
    """Two calls in a row on one input, y NaN-filled over the whole [2][pitch] row before
    each: y[:, :L] must match the render path, y[:, L:pitch] must be 0, and the caller's
    status word must keep its bits and gain no timeout bit."""
    import torch
    import paper_2408_03204_b300 as gx
    g = synth.Graph()
    i = g.add(synth.I)
    c = g.add(synth.C)
    o = g.add(synth.O)
    g.connect(i, c)
    g.connect(c, o)
    rpitch = (L + 3) // 4 * 4
    src_flat, _ = flat_sources([g], [L], [seed])
    P = {synth.C: np.array([[0.999, np.log(0.01), 0.6908, 5.0]], np.float32)}
    run = DeviceRun([g], [L], P, src_flat)   # ordinary path: grafx_render of i -> c -> o
    want = run.render().cpu().numpy().reshape(2, rpitch)
    u = torch.zeros(2, pitch, device="cuda")
    u[:, :rpitch] = run.src.view(2, rpitch)
    lib = gx.lib()
    stream = gx._stream(torch, run.src.device)
    status = torch.full((1,), status_init, dtype=torch.int32, device="cuda")
    for call in range(2):
        y = torch.full((2 * pitch,), float("nan"), device="cuda")
        rc = lib.grafx_compressor_forward_noalloc(ctypes.c_void_p(u.data_ptr()), L, pitch,
                                                  ctypes.c_void_p(run.P[synth.C].data_ptr()),
                                                  ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(status.data_ptr()),
                                                  stream)
        assert rc == 0, lib.grafx_last_error().decode()
        torch.cuda.synchronize()
        got = y.cpu().numpy().reshape(2, pitch)
        assert np.all(got[:, L:] == 0), f"call {call}: padding not zeroed"
        assert_out_close(got[:, :L], want[:, :L], tol=OUT_TOL)
        assert int(status.item()) == status_init, f"call {call}: status {int(status.item()):#x}"


def test_noalloc_compressor_matches_render_twice():
    L = 2 ** 17 + 6                       # 65 chunks, ragged tail
    _noalloc_vs_render(L, (L + 3) // 4 * 4, 31)


def test_noalloc_compressor_pads_far_past_the_last_chunk():
    # one chunk of 2048 samples covers the 100 samples; the row's pitch reaches 8192
    _noalloc_vs_render(100, 8192, 32, status_init=0x100)


def test_noalloc_compressor_rejects_oversized_input():
    import torch
    import paper_2408_03204_b300 as gx
    lib = gx.lib()
    x = torch.zeros(8, device="cuda")
    p = torch.tensor([0.99, 0.0, 0.7, 2.0], device="cuda")
    big = (1 << 22) + 1
    rc = lib.grafx_compressor_forward_noalloc(ctypes.c_void_p(x.data_ptr()), big, (big + 3) // 4 * 4,
                                              ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(x.data_ptr()), None,
                                              gx._stream(torch, x.device))
    assert gx.ERRORS.get(rc) == "ESHAPE"
    assert b"4194304" in lib.grafx_last_error()

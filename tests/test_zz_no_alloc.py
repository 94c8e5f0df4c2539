"""The allocation-free compressor call, for callers that must not allocate device memory
(real-time audio callbacks and plugin hosts, where an allocation can stall on a
device-wide synchronisation, and frameworks that own all device memory through their
own pool).  Its output must match the compressor of the ordinary render path on the
same input, on two calls in a row (the second call reuses the library's fixed scratch,
which the first call left dirty).

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


def test_noalloc_compressor_matches_render_twice():
    import torch
    import paper_2408_03204_b300 as gx
    g = synth.Graph()
    i = g.add(synth.I)
    c = g.add(synth.C)
    o = g.add(synth.O)
    g.connect(i, c)
    g.connect(c, o)
    L = 2 ** 17 + 6                       # 65 chunks, ragged tail
    pitch = (L + 3) // 4 * 4
    src_flat, _ = flat_sources([g], [L], [31])
    P = {synth.C: np.array([[0.999, np.log(0.01), 0.6908, 5.0]], np.float32)}
    run = DeviceRun([g], [L], P, src_flat)   # ordinary path: grafx_render of i -> c -> o
    want = run.render().cpu().numpy().reshape(2, pitch)
    lib = gx.lib()
    stream = gx._stream(torch, run.src.device)
    for call in range(2):
        y = torch.full((2 * pitch,), float("nan"), device="cuda")
        rc = lib.grafx_compressor_forward_noalloc(ctypes.c_void_p(run.src.data_ptr()), L, pitch,
                                                  ctypes.c_void_p(run.P[synth.C].data_ptr()),
                                                  ctypes.c_void_p(y.data_ptr()), stream)
        assert rc == 0, lib.grafx_last_error().decode()
        torch.cuda.synchronize()
        got = y.cpu().numpy().reshape(2, pitch)
        assert np.all(got[:, L:] == 0), f"call {call}: padding not zeroed"
        assert_out_close(got[:, :L], want[:, :L], tol=OUT_TOL)


def test_noalloc_compressor_rejects_oversized_input():
    import torch
    import paper_2408_03204_b300 as gx
    lib = gx.lib()
    x = torch.zeros(8, device="cuda")
    p = torch.tensor([0.99, 0.0, 0.7, 2.0], device="cuda")
    big = (1 << 22) + 1
    rc = lib.grafx_compressor_forward_noalloc(ctypes.c_void_p(x.data_ptr()), big, (big + 3) // 4 * 4,
                                              ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                              gx._stream(torch, x.device))
    assert gx.ERRORS.get(rc) == "ESHAPE"
    assert b"4194304" in lib.grafx_last_error()

"""Failure detection without a GPU fault: a bounded device wait on a flag that nothing
sets expires, records ST_TIMEOUT in the status word and returns; the context stays
usable.  Plans report such a word as GRAFX_ETIMEOUT through grafx_sync_status."""
import struct

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_bounded_wait_expires_and_reports():
    import torch
    import paper_2408_03204_b300 as gx
    lib = gx.lib()
    st = gx._stream(torch, torch.device("cuda"))
    flag = torch.zeros(1, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    value = torch.full((1,), 7.0, device="cuda")
    gx._check(lib.grafx_selftest_bounded_wait(gx._ptr(flag), gx._ptr(status), 20000, gx._ptr(value), st))
    torch.cuda.synchronize()
    assert int(status.item()) == 1 and value.item() == 0.0
    # a set flag (inclusive status 2, value 1.5) is read without expiry
    bits = struct.unpack("<I", struct.pack("<f", 1.5))[0]
    flag.fill_((2 << 32) | bits)
    status.zero_()
    gx._check(lib.grafx_selftest_bounded_wait(gx._ptr(flag), gx._ptr(status), 20000, gx._ptr(value), st))
    torch.cuda.synchronize()
    assert int(status.item()) == 0 and value.item() == 1.5
    # the context is still usable afterwards
    x = torch.arange(8.0, device="cuda")
    assert float((x * 2).sum()) == 56.0


def test_selftest_rejects_bad_limits():
    import torch
    import paper_2408_03204_b300 as gx
    lib = gx.lib()
    flag = torch.zeros(1, dtype=torch.int64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    value = torch.zeros(1, device="cuda")
    rc = lib.grafx_selftest_bounded_wait(gx._ptr(flag), gx._ptr(status), 0, gx._ptr(value),
                                         gx._stream(torch, flag.device))
    assert gx.ERRORS.get(rc) == "EINVAL"

"""Training-state files (paper_2408_03204_b300.state) on the host: round trip of every
supported dtype and shape, header contents, corruption detection."""
import os

import numpy as np
import pytest
import torch

from paper_2408_03204_b300.state import load_state, save_state


def test_round_trip(tmp_path):
    g = torch.Generator().manual_seed(0)
    ts = {"a": torch.randn(3, 5, generator=g), "b": torch.arange(7, dtype=torch.int32),
          "c": torch.randn(2, 2, generator=g).double(), "d": torch.tensor([1, -2], dtype=torch.int8),
          "e": torch.zeros(0, 4), "f": torch.randn(9, generator=g).to(torch.bfloat16), "g": torch.tensor(3)}
    p = os.path.join(tmp_path, "s.bin")
    save_state(p, ts, {"k": 1, "name": "x"})
    out, meta = load_state(p)
    assert meta == {"k": 1, "name": "x"}
    for k, v in ts.items():
        assert out[k].dtype == v.dtype and tuple(out[k].shape) == tuple(v.shape)
        assert torch.equal(out[k], v)


def test_offsets_aligned_and_truncation_detected(tmp_path):
    import json, struct
    p = os.path.join(tmp_path, "s.bin")
    save_state(p, {"a": torch.ones(3), "b": torch.ones(5, dtype=torch.int64)})
    raw = open(p, "rb").read()
    (h,) = struct.unpack("<Q", raw[8:16])
    header = json.loads(raw[16:16 + h])
    assert all(e["offset"] % 64 == 0 for e in header["tensors"])
    open(p, "wb").write(raw[:-4])
    with pytest.raises(ValueError):
        load_state(p)
    open(p, "wb").write(b"NOTSTATE" + raw[8:])
    with pytest.raises(ValueError):
        load_state(p)

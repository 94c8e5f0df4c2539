"""Training state on disk (fit and warm-start resume): one file holding a JSON header and
the raw bytes of named tensors.

Layout: 8 bytes magic ``GRAFXST1``, 8 bytes little-endian header length H, H bytes of
UTF-8 JSON ``{"meta": {...}, "tensors": [{"name", "dtype", "shape", "offset", "nbytes"}]}``,
then the tensor bytes, each starting at a 64-byte aligned offset from the start of the
data section.  Tensors are written from and read back to their own dtype and shape.
"""
import json
import struct

MAGIC = b"GRAFXST1"
_DTYPES = ("float32", "float64", "int32", "int64", "int8", "uint8", "bfloat16")


def save_state(path, tensors, meta=None):
    """tensors: {name: torch tensor (any device)}; meta: JSON-serialisable dict."""
    import torch
    entries, blobs, off = [], [], 0
    for name, t in tensors.items():
        dt = str(t.dtype).replace("torch.", "")
        if dt not in _DTYPES:
            raise ValueError(f"unsupported dtype {dt} for {name}")
        raw = t.detach().contiguous().cpu()
        data = raw.reshape(-1).view(torch.uint8).numpy().tobytes() if raw.numel() else b""
        pad = (-off) % 64
        off += pad
        blobs.append(b"\0" * pad + data)
        entries.append({"name": name, "dtype": dt, "shape": list(raw.shape), "offset": off, "nbytes": len(data)})
        off += len(data)
    header = json.dumps({"meta": meta or {}, "tensors": entries}).encode()
    with open(path, "wb") as f:
        f.write(MAGIC)
        f.write(struct.pack("<Q", len(header)))
        f.write(header)
        for b in blobs:
            f.write(b)


def load_state(path, device="cpu"):
    """Returns ({name: tensor on device}, meta)."""
    import numpy as np
    import torch
    with open(path, "rb") as f:
        if f.read(8) != MAGIC:
            raise ValueError(f"{path}: not a training-state file")
        (hlen,) = struct.unpack("<Q", f.read(8))
        header = json.loads(f.read(hlen).decode())
        data = f.read()
    out = {}
    for e in header["tensors"]:
        dt = getattr(torch, e["dtype"])
        buf = data[e["offset"]:e["offset"] + e["nbytes"]]
        if len(buf) != e["nbytes"]:
            raise ValueError(f"{path}: truncated tensor {e['name']}")
        t = torch.from_numpy(np.frombuffer(buf, dtype=np.uint8).copy())
        t = (t.view(dt) if len(buf) else torch.zeros(0, dtype=dt)).reshape(e["shape"])
        out[e["name"]] = t.to(device)
    return out, header["meta"]

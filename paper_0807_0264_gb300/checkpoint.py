"""Checkpoints of fields: one JSON header line, then the raw little-endian
bytes of each array.

The arrays are the library's own device layout (links (nfields, 4, 2, 9, Vh,
2), transforms (nfields, 2, 9, Vh, 2), FP64 or FP32; center sectors int8), so
a checkpoint is written and read without any conversion.  A relaxation
resumes from (U, Omega) alone: mcg_fix recomputes R at the start of every
call and counts sweeps from there, so a plain FP64 fix cut into calls of a
multiple of `reunit_every` sweeps, with a save and a load between them, gives
the links and the transform of one uninterrupted call bit for bit (the
relaxation is a fixed sequence of half-sweeps, Sec. II.A).

File layout:
    {"format": "mcg-fields", "version": 1, "dims": [Nx, Ny, Nz, Nt],
     "arrays": [{"name", "dtype", "shape", "offset", "nbytes"}, ...],
     "meta": {...}}\\n
    <raw bytes>
Offsets count from the first byte after the header line; dtypes are numpy
strings with explicit byte order ("<f8", "<f4", "|i1").
"""
from __future__ import annotations

import json

import numpy as np

FORMAT = "mcg-fields"
VERSION = 1
_DTYPES = {"float64": "<f8", "float32": "<f4", "int8": "|i1", "complex128": "<c16"}


def save(path, dims, arrays: dict, meta: dict | None = None) -> dict:
    """Write the named arrays (torch tensors on any device, or numpy arrays)
    and the JSON-serialisable `meta` to `path`.  Returns the header."""
    blobs, entries, off = [], [], 0
    for name, a in arrays.items():
        x = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
        dt = _DTYPES.get(x.dtype.name)
        if dt is None:
            raise TypeError(f"array {name!r}: unsupported dtype {x.dtype}")
        b = np.ascontiguousarray(x, dtype=np.dtype(dt)).tobytes()
        entries.append({"name": name, "dtype": dt, "shape": list(x.shape), "offset": off, "nbytes": len(b)})
        blobs.append(b)
        off += len(b)
    header = {"format": FORMAT, "version": VERSION, "dims": [int(d) for d in dims], "arrays": entries,
              "meta": meta or {}}
    with open(path, "wb") as f:
        f.write((json.dumps(header) + "\n").encode())
        for b in blobs:
            f.write(b)
    return header


def load(path, device=None):
    """Read a checkpoint: returns (header, {name: array}); the arrays are torch
    tensors on `device` when one is given, numpy arrays otherwise."""
    with open(path, "rb") as f:
        line = f.readline()
        try:
            header = json.loads(line)
        except ValueError as e:
            raise ValueError(f"{path}: not an {FORMAT} checkpoint") from e
        if header.get("format") != FORMAT or header.get("version") != VERSION:
            raise ValueError(f"{path}: not an {FORMAT} v{VERSION} checkpoint")
        data = f.read()
    out = {}
    for e in header["arrays"]:
        if e["offset"] + e["nbytes"] > len(data):
            raise ValueError(f"{path}: array {e['name']!r} is truncated")
        x = np.frombuffer(data, dtype=np.dtype(e["dtype"]), count=int(np.prod(e["shape"], dtype=np.int64)),
                          offset=e["offset"]).reshape(e["shape"])
        x = x.astype(x.dtype.newbyteorder("="), copy=True)
        if device is not None:
            import torch

            x = torch.from_numpy(x).to(device)
        out[e["name"]] = x
    return header, out

"""Content digests of CSR arrays (test helper; no method arithmetic).

A digest is the SHA-256 of the little-endian bytes of the row offsets
(int64), then the column ids (uint32), then the weights (float32) if any.
Stored expected values under tests/golden/ are digests of oracle outputs;
the GPU tests hash the library's downloaded output the same way.
"""
from __future__ import annotations

import hashlib

import numpy as np


def csr_digest(off, col, w=None) -> str:
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(off, dtype="<i8").tobytes())
    h.update(np.ascontiguousarray(np.asarray(col).view(np.uint32), dtype="<u4").tobytes())
    if w is not None:
        h.update(np.ascontiguousarray(w, dtype="<f4").tobytes())
    return h.hexdigest()


def read_golden(path: str) -> dict:
    """Parse a golden file: '#' comments, then 'key value...' lines."""
    out = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = vals
    return out

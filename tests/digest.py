"""Digests of whole k-mer histograms and of read sets, for comparing results too large to
keep side by side (test infrastructure; shares nothing with the oracle or the library).

A histogram's digest is the SHA-256 of its entries in ascending key order, each entry the
key's words as little-endian uint64 (the low word first for 128-bit keys) followed by
its count as a little-endian uint32."""
from __future__ import annotations

import hashlib

import numpy as np

CHUNK = 1 << 24  # entries packed per hash update


def _packed(keys: np.ndarray, counts: np.ndarray) -> np.ndarray:
    n = counts.shape[0]
    if keys.ndim == 1:
        out = np.empty(n, dtype=np.dtype([("k", "<u8"), ("c", "<u4")]))  # 12 bytes, packed
        out["k"] = keys
    else:
        out = np.empty(n, dtype=np.dtype([("lo", "<u8"), ("hi", "<u8"), ("c", "<u4")]))  # 20 bytes
        out["lo"] = keys[:, 0]
        out["hi"] = keys[:, 1]
    out["c"] = counts
    return out


class HistogramHasher:
    """Streaming digest: update() with consecutive ascending pieces of one histogram."""

    def __init__(self):
        self.h = hashlib.sha256()
        self.n = 0
        self.total = 0

    def update(self, keys: np.ndarray, counts: np.ndarray):
        for a in range(0, counts.shape[0], CHUNK):
            b = min(counts.shape[0], a + CHUNK)
            self.h.update(_packed(keys[a:b], counts[a:b]).tobytes())
        self.n += int(counts.shape[0])
        self.total += int(counts.sum(dtype=np.uint64))

    def hexdigest(self) -> str:
        return self.h.hexdigest()


def histogram_digest(keys: np.ndarray, counts: np.ndarray) -> str:
    hh = HistogramHasher()
    hh.update(keys, counts)
    return hh.hexdigest()


def input_digest(reads: np.ndarray, offsets: np.ndarray) -> str:
    """SHA-256 of the offsets (little-endian uint64) followed by the read bytes."""
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(offsets, dtype="<u8").tobytes())
    h.update(np.ascontiguousarray(reads, dtype=np.uint8).tobytes())
    return h.hexdigest()

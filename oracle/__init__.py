"""TEST INFRASTRUCTURE ONLY - the CPU oracle for the k-mer counter.

Only tests/, the smoke check in __graft_entry__ and the CPU-baseline leg of
bench.py may import this package.  The product library never does, and this
package never imports the product.

kc_oracle.c is the plain counter (Section II problem statement, Algorithm 1:
collect, Sort, Accumulate); brute.py is a string-based counter for tiny inputs
that pins it.  Both are written from the definition, independently of the GPU path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kc_oracle.c")
_LIB = os.path.join(_HERE, "libkc_oracle.so")

OR_OK, OR_EINVAL, OR_ENOMEM, OR_EOVERFLOW = 0, 1, 2, 4


class _Result(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("key_words", ctypes.c_uint32),
                ("keys", ctypes.c_void_p), ("counts", ctypes.c_void_p),
                ("n_valid_windows", ctypes.c_uint64)]


def build(force: bool = False) -> str:
    """Compile kc_oracle.c into libkc_oracle.so beside it."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, u64, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
        lib.oracle_count.argtypes = [vp, vp, u64, i32, i32, ctypes.POINTER(_Result)]
        lib.oracle_count.restype = i32
        lib.oracle_free.argtypes = [ctypes.POINTER(_Result)]
        lib.oracle_free.restype = None
        lib.oracle_valid_windows.argtypes = [vp, vp, u64, i32]
        lib.oracle_valid_windows.restype = u64
        lib.oracle_count_keys.argtypes = [vp, vp, u64, i32, i32, vp, u64, vp]
        lib.oracle_count_keys.restype = i32
        _lib = lib
    return _lib


def _ptrs(reads, offsets):
    reads = np.ascontiguousarray(reads, dtype=np.uint8)
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    return reads, offsets, len(offsets) - 1


def count(reads, offsets, k: int, canonical: bool = True):
    """Sorted histogram of the k-mers of the reads.

    Returns (keys, counts, n_valid_windows): keys uint64[n] for k <= 32 or
    uint64[n, 2] as (lo, hi) words for k > 32, ascending; counts uint32[n]."""
    lib = _load()
    reads, offsets, n = _ptrs(reads, offsets)
    res = _Result()
    rc = lib.oracle_count(reads.ctypes.data, offsets.ctypes.data, n, int(k), int(bool(canonical)), ctypes.byref(res))
    if rc not in (OR_OK,):
        lib.oracle_free(ctypes.byref(res))
        raise ValueError(f"oracle_count failed with status {rc}")
    try:
        d, kw = int(res.n), int(res.key_words)
        keys = np.empty(d * kw, dtype=np.uint64)
        counts = np.empty(d, dtype=np.uint32)
        if d:
            ctypes.memmove(keys.ctypes.data, res.keys, 8 * d * kw)
            ctypes.memmove(counts.ctypes.data, res.counts, 4 * d)
        if kw == 2:
            keys = keys.reshape(d, 2)
        return keys, counts, int(res.n_valid_windows)
    finally:
        lib.oracle_free(ctypes.byref(res))


def valid_windows(reads, offsets, k: int) -> int:
    """Number of windows of k bases (ACGTacgt only) inside one read."""
    reads, offsets, n = _ptrs(reads, offsets)
    return int(_load().oracle_valid_windows(reads.ctypes.data, offsets.ctypes.data, n, int(k)))


def count_keys(reads, offsets, k: int, canonical: bool, query) -> np.ndarray:
    """Occurrences of each queried key (ascending, distinct) among all windows."""
    reads, offsets, n = _ptrs(reads, offsets)
    q = np.ascontiguousarray(query, dtype=np.uint64)
    nq = q.shape[0]
    out = np.zeros(nq, dtype=np.uint64)
    rc = _load().oracle_count_keys(reads.ctypes.data, offsets.ctypes.data, n, int(k), int(bool(canonical)),
                                   q.ctypes.data, nq, out.ctypes.data)
    if rc:
        raise ValueError(f"oracle_count_keys failed with status {rc}")
    return out


def count_parallel(reads, offsets, k: int, canonical: bool = True, threads: int | None = None):
    """The same histogram as count(), computed on several host cores: the reads are cut into
    `threads` ranges, each counted by count() in its own thread (the C call releases the
    GIL), and the sorted per-range histograms are merged by key with their counts added
    (counting is additive over disjoint read sets), the merge itself split into key ranges
    that threads sort and sum apart.  This is the multi-threaded CPU variant timed beside
    the GPU; count() stays the reference definition.

    Returns (keys, counts, n_valid_windows) like count()."""
    import concurrent.futures as cf
    threads = max(1, int(threads or os.cpu_count() or 1))
    offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
    n = len(offsets) - 1
    cuts = np.linspace(0, n, threads + 1).astype(np.int64)
    kw = 1 if k <= 32 else 2

    def part(i):
        a, b = int(cuts[i]), int(cuts[i + 1])
        keys, counts, nv = count(reads[int(offsets[a]):int(offsets[b])], offsets[a:b + 1] - offsets[a], k, canonical)
        return keys.reshape(-1, kw), counts, nv

    with cf.ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(part, range(threads)))
    windows = sum(p[2] for p in parts)
    # key ranges cut on the top key word, at quantiles of a sample of the keys
    tops = [p[0][:, kw - 1] for p in parts]
    sample = np.concatenate([t[:: max(1, t.size // 1024)] for t in tops]) if tops else np.zeros(0, np.uint64)
    pivots = np.unique(np.quantile(sample.astype(np.float64), np.linspace(0, 1, threads + 1)[1:-1])
                       .astype(np.uint64)) if sample.size else np.zeros(0, np.uint64)
    bounds = [np.concatenate([[0], np.searchsorted(t, pivots, side="left"), [t.size]]) for t in tops]

    def merge(r):
        keys = np.concatenate([p[0][int(b[r]):int(b[r + 1])] for p, b in zip(parts, bounds)])
        counts = np.concatenate([p[1][int(b[r]):int(b[r + 1])] for p, b in zip(parts, bounds)]).astype(np.uint64)
        if counts.size == 0:
            return keys, counts
        order = np.lexsort((keys[:, 0], keys[:, 1])) if kw == 2 else np.argsort(keys[:, 0], kind="stable")
        keys = keys[order]
        new = np.ones(counts.size, dtype=bool)
        new[1:] = np.any(keys[1:] != keys[:-1], axis=1)
        starts = np.flatnonzero(new)
        return keys[starts], np.add.reduceat(counts[order], starts)

    with cf.ThreadPoolExecutor(threads) as ex:
        merged = list(ex.map(merge, range(len(pivots) + 1)))
    keys = np.concatenate([m[0] for m in merged]) if merged else np.zeros((0, kw), np.uint64)
    counts = np.concatenate([m[1] for m in merged]) if merged else np.zeros(0, np.uint64)
    if counts.size and counts.max() > 0xFFFFFFFF:
        raise ValueError("a count exceeds 2^32 - 1")
    return (keys.reshape(-1) if kw == 1 else keys), counts.astype(np.uint32), windows

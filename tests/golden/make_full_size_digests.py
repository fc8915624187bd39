"""Write tests/golden/full_size_digests.json: the SHA-256 of the whole sorted histogram of
each full-size workload, computed by the CPU oracle alone (nothing from the CUDA path).

    python tests/golden/make_full_size_digests.py [--threads N] [workload ...]

The oracle counts one read range at a time (oracle.count: every window's key from its own
k bytes, qsort, run-length encode; Section II, Algorithm 1).  Counting is additive over
disjoint read sets (pinned in tests/test_oracle.py), so the histogram of all reads is the
per-range histograms merged by key with their counts added.  The merge goes key range by
key range (ranges cut on the top key word), each range's pieces sorted together and equal
keys summed, and the ascending result streams into the digest of tests/digest.py.  The
input's own digest is stored beside it, so that a test can tell whether it generated the
same reads.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402
from tests.digest import HistogramHasher, input_digest  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "full_size_digests.json")
WORKLOADS = ["repeats_100mbp_150bp_30x_k31", "long_50mbp_10kbp_20x_k63"]


def chunk_histograms(reads, offsets, k, canonical, n_chunks, threads):
    """oracle.count of each of n_chunks read ranges (threads: the C call releases the GIL)."""
    n = len(offsets) - 1
    cuts = np.linspace(0, n, n_chunks + 1).astype(np.int64)

    def part(i):
        a, b = int(cuts[i]), int(cuts[i + 1])
        o = offsets[a:b + 1] - offsets[a]
        r = reads[int(offsets[a]):int(offsets[b])]
        return oracle.count(r, o, k, canonical)

    with cf.ThreadPoolExecutor(threads) as ex:
        return list(ex.map(part, range(n_chunks)))


def top_word(keys):
    return keys if keys.ndim == 1 else keys[:, 1]


def merged_digest(parts, n_ranges=64):
    """Digest of the sum of the sorted histograms `parts` (list of (keys, counts, windows)),
    merged one top-word range at a time.  Returns (digest, distinct keys, windows)."""
    pivots_src = np.concatenate([top_word(p[0])[:: max(1, len(p[1]) // 4096)] for p in parts if len(p[1])])
    pivots = np.unique(np.quantile(pivots_src.astype(np.float64), np.linspace(0, 1, n_ranges + 1)[1:-1]).astype(np.uint64)) \
        if pivots_src.size else np.zeros(0, np.uint64)
    bounds = [np.concatenate([[0], np.searchsorted(top_word(p[0]), pivots, side="left"), [len(p[1])]]) for p in parts]
    hh = HistogramHasher()
    for r in range(len(pivots) + 1):
        ks = [p[0][int(b[r]):int(b[r + 1])] for p, b in zip(parts, bounds)]
        cs = [p[1][int(b[r]):int(b[r + 1])] for p, b in zip(parts, bounds)]
        keys = np.concatenate(ks) if ks else np.zeros(0, np.uint64)
        counts = np.concatenate(cs).astype(np.uint64) if cs else np.zeros(0, np.uint64)
        if counts.size == 0:
            continue
        if keys.ndim == 1:
            order = np.argsort(keys, kind="stable")
            keys = keys[order]
            new = np.ones(keys.size, dtype=bool)
            new[1:] = keys[1:] != keys[:-1]
        else:
            order = np.lexsort((keys[:, 0], keys[:, 1]))  # by high word, then low word
            keys = keys[order]
            new = np.ones(keys.shape[0], dtype=bool)
            new[1:] = (keys[1:, 0] != keys[:-1, 0]) | (keys[1:, 1] != keys[:-1, 1])
        counts = counts[order]
        starts = np.flatnonzero(new)
        summed = np.add.reduceat(counts, starts)
        if summed.max() > 0xFFFFFFFF:
            raise OverflowError("a count exceeds 2^32 - 1")
        hh.update(keys[starts], summed.astype(np.uint32))
    return hh.hexdigest(), hh.n, hh.total


def oracle_full_digest(reads, offsets, k, canonical=True, threads=None, n_chunks=32):
    threads = threads or os.cpu_count() or 4
    parts = chunk_histograms(reads, offsets, k, canonical, n_chunks, threads)
    windows = sum(p[2] for p in parts)
    digest, distinct, total = merged_digest(parts)
    if total != windows:
        raise RuntimeError(f"merged counts {total} != windows {windows}")
    return {"sha256": digest, "distinct": distinct, "windows": windows}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("workloads", nargs="*", default=WORKLOADS)
    args = ap.parse_args()
    out = {}
    if os.path.exists(OUT):
        with open(OUT) as f:
            out = json.load(f)
    for name in args.workloads:
        t0 = time.time()
        reads, offsets, k = synth.workload(name)
        d = oracle_full_digest(reads, offsets, k, True, args.threads or None)
        d.update({"k": k, "canonical": True, "reads": len(offsets) - 1, "bases": int(offsets[-1]),
                  "input_sha256": input_digest(reads, offsets),
                  "command": "python tests/golden/make_full_size_digests.py " + name})
        out[name] = d
        print(name, d, f"{time.time() - t0:.0f} s", flush=True)
        with open(OUT, "w") as f:
            json.dump(out, f, indent=1, sort_keys=True)


if __name__ == "__main__":
    main()

"""Golden fixtures (text) and their loader."""
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))


def aatgg_repeat():
    """(reads, offsets, {(canonical, k): (keys, counts)}) of tests/golden/aatgg_repeat.txt."""
    table = {}
    with open(os.path.join(HERE, "aatgg_repeat.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            mode, k, key, count = line.split()[:4]
            table.setdefault((mode == "canonical", int(k)), []).append((int(key), int(count)))
    reads = np.frombuffer(b"AATGG" * 20, dtype=np.uint8).copy()
    offsets = np.array([0, reads.size], dtype=np.uint64)
    out = {}
    for key, rows in table.items():
        rows.sort()
        out[key] = (np.array([r[0] for r in rows], np.uint64), np.array([r[1] for r in rows], np.uint32))
    return reads, offsets, out

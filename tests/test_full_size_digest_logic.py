"""The full-size digest recipe (tests/golden/make_full_size_digests.py) on inputs small
enough for one oracle call: counting read ranges apart and merging them key range by key
range gives exactly the digest of the oracle's histogram of all the reads."""
import numpy as np
import pytest

import oracle
import synth
from tests.digest import histogram_digest, input_digest
from tests.golden.make_full_size_digests import oracle_full_digest


@pytest.mark.parametrize("gen,seed,scale,k", [
    (synth.REPEAT_SHORT, 1002, 0.002, 31),   # heavy repeats, 64-bit keys
    (synth.LONG_NOISY, 1003, 0.001, 63),     # long noisy reads, 128-bit keys
    (synth.UNIFORM_SHORT, 1001, 0.05, 21),
])
def test_chunked_merge_equals_one_count(gen, seed, scale, k):
    reads, offsets, _ = synth.generate(gen, seed, scale)
    keys, counts, nv = oracle.count(reads, offsets, k, True)
    want = histogram_digest(keys, counts)
    got = oracle_full_digest(reads, offsets, k, True, threads=4, n_chunks=7)
    assert got == {"sha256": want, "distinct": len(counts), "windows": nv}


def test_digest_sees_a_swapped_count_and_a_changed_key():
    keys = np.array([3, 5, 9], np.uint64)
    counts = np.array([1, 2, 3], np.uint32)
    d = histogram_digest(keys, counts)
    assert histogram_digest(keys, counts[[0, 2, 1]]) != d
    assert histogram_digest(np.array([3, 6, 9], np.uint64), counts) != d
    k2 = np.array([[3, 0], [5, 1]], np.uint64)
    assert histogram_digest(k2, counts[:2]) != histogram_digest(k2[:, ::-1].copy(), counts[:2])


def test_input_digest_depends_on_reads_and_offsets():
    r = np.frombuffer(b"ACGTACGT", np.uint8)
    assert input_digest(r, np.array([0, 8], np.uint64)) != input_digest(r, np.array([0, 4, 8], np.uint64))

"""Pins for the CPU oracle (oracle/kc_oracle.c), none of which re-derive its code:
a string-level brute force, hand-worked examples, closed forms (homopolymers,
de Bruijn sequences), invariants of the exact histogram, and a mutation check
that plants plausible mistakes in a copy of the oracle and sees a pin fail."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import synth
from oracle import brute
from tests.kmer_math import keys_as_ints, rc_key, key_to_str

KS = [1, 2, 3, 4, 5, 8, 15, 16, 17, 31, 32, 33, 47, 63, 64]


def as_reads(strings):
    bs = [s.encode() if isinstance(s, str) else s for s in strings]
    offsets = np.zeros(len(bs) + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum([len(b) for b in bs])
    reads = np.frombuffer(b"".join(bs), dtype=np.uint8).copy() if bs else np.zeros(0, np.uint8)
    return reads, offsets


def oracle_pairs(reads, offsets, k, canonical):
    keys, counts, _ = oracle.count(reads, offsets, k, canonical)
    return list(zip(keys_as_ints(keys), [int(c) for c in counts]))


def split_reads(reads, offsets):
    return [bytes(reads[int(offsets[i]):int(offsets[i + 1])]) for i in range(len(offsets) - 1)]


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("seed", range(6))
def test_oracle_matches_string_brute_force(seed):
    rng = np.random.default_rng(seed)
    reads, offsets = synth.random_reads(rng, n_reads=int(rng.integers(0, 40)), max_len=80)
    rs = split_reads(reads, offsets)
    for k in KS:
        for canonical in (False, True):
            assert oracle_pairs(reads, offsets, k, canonical) == brute.sorted_histogram(rs, k, canonical), (k, canonical)


# ---------------------------------------------------------------- worked examples (derived by hand)
def test_worked_example_acgt_k2():
    # ACGT, k=2: windows AC(=0*4+1=1) CG(=1*4+2=6) GT(=2*4+3=11).
    # reverse complements: AC->GT, CG->CG (palindrome), GT->AC.
    # canonical: AC:min(1,11)=1, CG:6, GT:min(11,1)=1  => {1:2, 6:1}
    r, o = as_reads(["ACGT"])
    assert oracle_pairs(r, o, 2, True) == [(1, 2), (6, 1)]
    assert oracle_pairs(r, o, 2, False) == [(1, 1), (6, 1), (11, 1)]


def test_worked_example_read_boundary_and_n():
    # reads "AC" and "GT" are adjacent in memory; "CG" spans the boundary and must not count.
    r, o = as_reads(["AC", "GT"])
    assert oracle_pairs(r, o, 2, False) == [(1, 1), (11, 1)]
    assert oracle_pairs(r, o, 2, True) == [(1, 2)]
    # "ACNGT", k=2: AC and GT count, CN and NG do not.
    r, o = as_reads(["ACNGT"])
    assert oracle_pairs(r, o, 2, False) == [(1, 1), (11, 1)]
    # lowercase reads count as uppercase: "acgt" == "ACGT"
    r, o = as_reads(["acgt"])
    assert oracle_pairs(r, o, 2, True) == [(1, 2), (6, 1)]


def test_worked_example_k1():
    # k=1 canonical: A,T -> 0 (A);  C,G -> 1 (C)
    r, o = as_reads(["AACGTTT"])
    assert oracle_pairs(r, o, 1, True) == [(0, 5), (1, 2)]
    assert oracle_pairs(r, o, 1, False) == [(0, 2), (1, 1), (2, 1), (3, 3)]


def test_worked_example_word_edges():
    # k=32, all T, not canonical: 32 digits of 3 = 4^32 - 1 = 2^64 - 1 (every bit set)
    r, o = as_reads(["T" * 40])
    assert oracle_pairs(r, o, 32, False) == [(2**64 - 1, 9)]
    # canonical: TTT..T -> its reverse complement AAA..A = 0
    assert oracle_pairs(r, o, 32, True) == [(0, 9)]
    # k=64, all T, not canonical: 2^128 - 1
    r, o = as_reads(["T" * 64])
    assert oracle_pairs(r, o, 64, False) == [(2**128 - 1, 1)]
    # k=33: A^32 C -> forward = 1; reverse complement G T^32 = 2*4^32 + 4^32 - 1; min = 1
    r, o = as_reads(["A" * 32 + "C"])
    assert oracle_pairs(r, o, 33, True) == [(1, 1)]
    assert oracle_pairs(r, o, 33, False) == [(1, 1)]
    # k=33: C A^32 -> forward = 4^32 = 2^64 (first bit of the high word)
    r, o = as_reads(["C" + "A" * 32])
    assert oracle_pairs(r, o, 33, False) == [(2**64, 1)]


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("k", [1, 7, 31, 32, 33, 63, 64])
def test_homopolymer(k):
    m = 150
    r, o = as_reads(["A" * m])
    assert oracle_pairs(r, o, k, True) == [(0, m - k + 1)]
    r, o = as_reads(["T" * m])
    assert oracle_pairs(r, o, k, True) == [(0, m - k + 1)]
    assert oracle_pairs(r, o, k, False) == [(4**k - 1, m - k + 1)]


def de_bruijn(n: int) -> str:
    """B(4, n) by concatenating Lyndon words whose length divides n (FKM algorithm),
    linearised by appending its first n-1 symbols."""
    a = [0] * (n + 1)
    seq = []

    def gen(t, p):
        if t > n:
            if n % p == 0:
                seq.extend(a[1:p + 1])
        else:
            a[t] = a[t - p]
            gen(t + 1, p)
            for j in range(a[t - p] + 1, 4):
                a[t] = j
                gen(t + 1, t)

    gen(1, 1)
    s = "".join("ACGT"[d] for d in seq)
    return s + s[:n - 1]


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_de_bruijn_every_kmer_once(k):
    s = de_bruijn(k)
    assert len(s) == 4**k + k - 1
    r, o = as_reads([s])
    assert oracle_pairs(r, o, k, False) == [(v, 1) for v in range(4**k)]


def test_empty_inputs():
    r, o = as_reads([])
    assert oracle_pairs(r, o, 31, True) == []
    r, o = as_reads(["", "ACG", "N" * 50, ""])
    assert oracle_pairs(r, o, 4, True) == []
    r, o = as_reads(["ACGT"])
    assert oracle_pairs(r, o, 5, False) == []
    assert oracle_pairs(r, o, 4, False) == [(27, 1)]  # ACGT = 0*64+1*16+2*4+3


def test_invalid_arguments():
    r, o = as_reads(["ACGT"])
    for k in (0, 65, -1):
        with pytest.raises(ValueError):
            oracle.count(r, o, k, True)
    bad = np.array([0, 3, 2], dtype=np.uint64)
    with pytest.raises(ValueError):
        oracle.count(np.zeros(3, np.uint8), bad, 1, True)


# ---------------------------------------------------------------- invariants on workload-shaped inputs
def small_workloads():
    yield synth.generate(synth.UNIFORM_SHORT, 1001, 0.02)[:2], 31
    yield synth.generate(synth.REPEAT_SHORT, 1002, 0.0004)[:2], 31
    yield synth.generate(synth.LONG_NOISY, 1003, 0.0008)[:2], 63


def test_invariants_on_workload_shapes():
    for (reads, offsets), k in small_workloads():
        keys, counts, nv = oracle.count(reads, offsets, k, True)
        ints = keys_as_ints(keys)
        assert nv == oracle.valid_windows(reads, offsets, k) > 0
        assert int(counts.astype(np.uint64).sum()) == nv
        assert all(a < b for a, b in zip(ints, ints[1:]))
        assert counts.min() >= 1
        # canonical keys are the smaller of the pair (checked on a sample, digit by digit)
        for v in ints[:: max(1, len(ints) // 500)]:
            assert v <= rc_key(v, k)


def test_permutation_reverse_complement_and_additivity():
    (reads, offsets), k = next(small_workloads())
    rs = split_reads(reads, offsets)
    base = oracle_pairs(reads, offsets, k, True)
    rng = np.random.default_rng(7)
    perm = [rs[i] for i in rng.permutation(len(rs))]
    assert oracle_pairs(*as_reads(perm), k, True) == base
    comp = bytes.maketrans(b"ACGTacgt", b"TGCAtgca")
    rcs = [r.translate(comp)[::-1] for r in rs]
    assert oracle_pairs(*as_reads(rcs), k, True) == base
    h = len(rs) // 3
    a = dict(oracle_pairs(*as_reads(rs[:h]), k, True))
    for key, c in oracle_pairs(*as_reads(rs[h:]), k, True):
        a[key] = a.get(key, 0) + c
    assert sorted(a.items()) == base
    # canonical = forward histogram folded by min(key, rc(key))
    fold = {}
    for key, c in oracle_pairs(reads, offsets, k, False):
        m = min(key, rc_key(key, k))
        fold[m] = fold.get(m, 0) + c
    assert sorted(fold.items()) == base


def test_count_keys_agrees_with_count():
    for (reads, offsets), k in small_workloads():
        keys, counts, _ = oracle.count(reads, offsets, k, True)
        idx = np.unique(np.linspace(0, len(counts) - 1, 300).astype(np.int64))
        q = keys[idx]
        got = oracle.count_keys(reads, offsets, k, True, q)
        assert np.array_equal(got, counts[idx].astype(np.uint64))
        # a key that cannot occur: the all-T k-mer is never canonical (its rc is all-A)
        allt = (1 << (2 * k)) - 1
        qq = np.array([allt], dtype=np.uint64) if k <= 32 else np.array([[allt & (2**64 - 1), allt >> 64]], dtype=np.uint64)
        assert oracle.count_keys(reads, offsets, k, True, qq)[0] == 0


def test_key_string_helper_round_trip():
    assert key_to_str(27, 4) == "ACGT"
    assert rc_key(27, 4) == 27  # ACGT is its own reverse complement


# ---------------------------------------------------------------- planted mistakes must fail a pin
MUTATIONS = {
    "code order": ("case 'C': case 'c': return 1;", "case 'C': case 'c': return 2;"),
    "max not min": ("(canonical && rc < fwd)", "(canonical && rc > fwd)"),
    "no complement": ("(u128)(3 - base_code(w[t]))", "(u128)(base_code(w[t]))"),
    "rc not reversed": ("for (int t = k - 1; t >= 0; --t) rc", "for (int t = 0; t < k; ++t) rc"),
    "N kept": ("default: return -1;", "default: return 0;"),
    "last window dropped": ("j + (uint64_t)k <= len; ++j) {\n      u128 key;\n      if (window_key(r + j, k, canonical, &key) == 0)",
                            "j + (uint64_t)k < len; ++j) {\n      u128 key;\n      if (window_key(r + j, k, canonical, &key) == 0)"),
    "digits reversed": ("fwd = fwd * 4 + (u128)c;", "fwd = fwd + ((u128)c << (2 * t));"),
    "lowercase rejected": ("case 'A': case 'a': return 0;", "case 'A': return 0;"),
    "count off by one": ("out->counts[q] = (uint32_t)(j - i);", "out->counts[q] = (uint32_t)(j - i + (j - i > 1));"),
    "high word dropped": ("out->keys[2 * q + 1] = (uint64_t)(T[i] >> 64);", "out->keys[2 * q + 1] = 0;"),
}


def _mutant(tmp_path, name, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "kc_oracle.c")).read()
    assert src.count(old) >= 1, name
    path = tmp_path / f"m_{abs(hash(name))}.c"
    path.write_text(src.replace(old, new))
    so = str(path) + ".so"
    subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-o", so, str(path)])
    lib = ctypes.CDLL(so)
    lib.oracle_count.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(oracle._Result)]
    lib.oracle_count.restype = ctypes.c_int
    return lib


def _run(lib, reads, offsets, k, canonical):
    res = oracle._Result()
    reads = np.ascontiguousarray(reads, np.uint8)
    offsets = np.ascontiguousarray(offsets, np.uint64)
    lib.oracle_count(reads.ctypes.data, offsets.ctypes.data, len(offsets) - 1, k, int(canonical), ctypes.byref(res))
    d, kw = int(res.n), int(res.key_words)
    keys = np.ctypeslib.as_array(ctypes.cast(res.keys, ctypes.POINTER(ctypes.c_uint64)), (max(d * kw, 1),))[: d * kw].copy()
    counts = np.ctypeslib.as_array(ctypes.cast(res.counts, ctypes.POINTER(ctypes.c_uint32)), (max(d, 1),))[:d].copy()
    if kw == 2:
        keys = keys.reshape(d, 2)
    return list(zip(keys_as_ints(keys), [int(c) for c in counts]))


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTATIONS[name]
    lib = _mutant(tmp_path, name, old, new)
    rng = np.random.default_rng(11)
    reads, offsets = synth.random_reads(rng, n_reads=30, max_len=90)
    rs = split_reads(reads, offsets)
    caught = False
    for k in (2, 5, 31, 33, 64):
        for canonical in (False, True):
            if _run(lib, reads, offsets, k, canonical) != brute.sorted_histogram(rs, k, canonical):
                caught = True
    assert caught, f"pins did not catch planted mistake: {name}"


# ---------------------------------------------------------------- golden fixture
def test_golden_aatgg_repeat():
    """The paper's heavy-hitter repeat (AATGG)_n, Section IV-D: closed-form histogram."""
    from tests.golden import aatgg_repeat
    reads, offsets, want = aatgg_repeat()
    assert len(want) == 4
    for (canonical, k), (wk, wc) in want.items():
        keys, counts, nv = oracle.count(reads, offsets, k, canonical)
        assert np.array_equal(keys, wk) and np.array_equal(counts, wc), (canonical, k)
        assert nv == reads.size - k + 1


@pytest.mark.parametrize("k,canonical,threads", [(31, True, 4), (63, True, 3), (21, False, 7), (5, True, 16)])
def test_parallel_variant_equals_the_oracle(k, canonical, threads):
    """The multi-threaded variant (read ranges counted apart, merged by key with addition)
    gives exactly the single-threaded oracle's histogram."""
    reads, offsets, _ = synth.generate(synth.UNIFORM_SHORT, 1001, 0.02)
    want = oracle.count(reads, offsets, k, canonical)
    got = oracle.count_parallel(reads, offsets, k, canonical, threads)
    assert got[2] == want[2]
    assert np.array_equal(got[0], want[0]) and np.array_equal(got[1], want[1])

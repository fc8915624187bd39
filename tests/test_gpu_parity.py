"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer work: every comparison is bit-exact (keys and counts, byte for byte).
Small and medium inputs are compared in full; the full-size workloads through the
SHA-256 of the whole sorted histogram, against the oracle's."""
import os

import numpy as np
import pytest

import oracle
import synth


pytestmark = pytest.mark.gpu

KS = [1, 2, 3, 4, 5, 8, 15, 16, 17, 31, 32, 33, 47, 63, 64]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def counter(torch_cuda):
    from paper_2505_04431_gb300 import KmerCounter, build
    build.build()
    c = KmerCounter()
    yield c
    c.close()


def gpu_count(counter, reads, offsets, k, canonical):
    res = counter.count(reads, offsets, k, canonical)
    try:
        keys, counts = res.to_numpy()
        return keys, counts, res.n_valid_windows
    finally:
        res.free()


def assert_parity(counter, reads, offsets, k, canonical, tag=""):
    ok, oc, onv = oracle.count(reads, offsets, k, canonical)
    gk, gc, gnv = gpu_count(counter, reads, offsets, k, canonical)
    assert gnv == onv, f"{tag} valid windows {gnv} != {onv}"
    assert gk.shape == ok.shape, f"{tag} distinct {gk.shape} != {ok.shape}"
    assert np.array_equal(gk, ok), f"{tag} keys differ"
    assert np.array_equal(gc, oc), f"{tag} counts differ"


def as_reads(strings):
    bs = [s.encode() if isinstance(s, str) else s for s in strings]
    offsets = np.zeros(len(bs) + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum([len(b) for b in bs])
    reads = np.frombuffer(b"".join(bs), dtype=np.uint8).copy() if bs else np.zeros(0, np.uint8)
    return reads, offsets


# ---------------------------------------------------------------- small random inputs, every k
@pytest.mark.parametrize("seed", range(4))
def test_random_small_all_k(counter, seed):
    rng = np.random.default_rng(100 + seed)
    reads, offsets = synth.random_reads(rng, n_reads=int(rng.integers(1, 300)), max_len=200)
    for k in KS:
        for canonical in (False, True):
            assert_parity(counter, reads, offsets, k, canonical, f"seed={seed} k={k} c={canonical}")


def test_random_many_reads_cross_tiles(counter):
    # ~1.3 M bases: several 262144-base tiles, reads straddle tile and word boundaries
    rng = np.random.default_rng(7)
    reads, offsets = synth.random_reads(rng, n_reads=9000, max_len=300, junk=0.001, n_rate=0.002)
    for k in (21, 31, 32, 33, 63, 64):
        assert_parity(counter, reads, offsets, k, True, f"k={k}")
    assert_parity(counter, reads, offsets, 32, False, "k=32 fwd")
    assert_parity(counter, reads, offsets, 64, False, "k=64 fwd")


# ---------------------------------------------------------------- workload-shaped inputs
@pytest.mark.parametrize("name,gen,seed,scale,k", [
    ("uniform 1 Mbp 100 bp 10x", synth.UNIFORM_SHORT, 1001, 1.0, 31),
    ("repeats 0.5 Mbp 150 bp 30x", synth.REPEAT_SHORT, 1002, 0.005, 31),
    ("long noisy 1 Mbp 20x k63", synth.LONG_NOISY, 1003, 0.02, 63),
])
def test_workload_shapes(counter, name, gen, seed, scale, k):
    reads, offsets, _ = synth.generate(gen, seed, scale)
    assert_parity(counter, reads, offsets, k, True, name)


def test_workload_shapes_forward_and_other_k(counter):
    reads, offsets, _ = synth.generate(synth.UNIFORM_SHORT, 1001, 0.3)
    for k in (21, 31, 32):
        assert_parity(counter, reads, offsets, k, False, f"fwd k={k}")
    reads, offsets, _ = synth.generate(synth.LONG_NOISY, 1003, 0.005)
    for k in (33, 47, 64):
        assert_parity(counter, reads, offsets, k, True, f"long k={k}")


# ---------------------------------------------------------------- edge cases
def test_empty_and_degenerate(counter):
    for strings, k in [([], 31), ([""], 5), (["", "", ""], 1), (["ACG"], 4), (["N" * 500], 3),
                       (["ACGT"], 4), (["ACGTN" * 40], 4), (["A" * 31], 31), (["a" * 64], 64)]:
        r, o = as_reads(strings)
        for canonical in (False, True):
            assert_parity(counter, r, o, k, canonical, f"{strings[:1]} k={k}")


def test_heavy_hitter_single_key(counter):
    # 20000 identical homopolymer reads: one key with 2.42 M occurrences (all warp lanes equal)
    r, o = as_reads(["A" * 150] * 20000)
    ok, oc, _ = oracle.count(r, o, 31, True)
    assert oc.tolist() == [20000 * 120]
    assert_parity(counter, r, o, 31, True, "homopolymer")
    assert_parity(counter, r, o, 63, True, "homopolymer k63")
    # mixed: heavy key among random reads
    rng = np.random.default_rng(3)
    rr, ro = synth.random_reads(rng, n_reads=3000, max_len=150, junk=0.0, lower=0.0, n_rate=0.0)
    strings = [bytes(rr[int(ro[i]):int(ro[i + 1])]) for i in range(3000)] + [b"AC" * 75] * 3000
    r, o = as_reads(strings)
    for k in (8, 31, 33):
        assert_parity(counter, r, o, k, True, f"mixed heavy k={k}")


def test_keys_clumped_under_a_long_prefix(counter):
    # reads that open with a long A run and go on at random: thousands of distinct canonical
    # keys share their leading zero bits, so within the first partition they fall in a
    # handful of order buckets far above average size (sorted by a warp, not ranked by
    # counting), and the partition overflows its table (split into key sub-ranges)
    rng = np.random.default_rng(11)
    bases = np.frombuffer(b"ACGT", dtype=np.uint8)
    strings = []
    for i in range(4000):
        tail = bases[rng.integers(0, 4, size=int(rng.integers(20, 60)))].tobytes()
        strings.append(b"A" * int(rng.integers(20, 40)) + tail)
        if i % 4 == 0:  # the reverse-complement form of the same clump
            strings.append(tail[::-1].translate(bytes.maketrans(b"ACGT", b"TGCA")) + b"T" * 30)
    r, o = as_reads(strings)
    for k in (21, 31, 33, 63):
        assert_parity(counter, r, o, k, True, f"clumped k={k}")
    assert_parity(counter, r, o, 31, False, "clumped fwd k=31")


def test_all_ones_key(counter):
    # non-canonical k=32 / k=64: the all-T k-mer has every key bit set
    for k in (32, 64):
        r, o = as_reads(["T" * 100, "ACGT" * 30, "T" * k, "GGT" + "T" * 70])
        assert_parity(counter, r, o, k, False, f"all-T k={k}")
        assert_parity(counter, r, o, k, True, f"all-T canonical k={k}")


def test_reads_exactly_k_and_tile_boundaries(counter):
    # reads of exactly k bases; read starts placed at and next to the 262144-base tile boundary
    rng = np.random.default_rng(5)
    seqs = []
    total = 0
    while total < 262144 - 40:
        n = int(rng.integers(1, 200))
        seqs.append("".join("ACGT"[i] for i in rng.integers(0, 4, n)))
        total += n
    seqs.append("C" * (262144 - total))  # next read starts exactly at the boundary
    seqs += ["".join("ACGT"[i] for i in rng.integers(0, 4, 31)) for _ in range(3000)]
    r, o = as_reads(seqs)
    assert int(o[len(seqs) - 3000]) == 262144
    assert_parity(counter, r, o, 31, True, "exact-k reads")
    assert_parity(counter, r, o, 5, False, "exact-k reads k5")


def test_overflow_path_forced(torch_cuda):
    # tiny tables: nearly every fine partition overflows and is split by key range
    from paper_2505_04431_gb300 import KmerCounter
    c = KmerCounter(table_slots_max=64)
    try:
        reads, offsets, _ = synth.generate(synth.UNIFORM_SHORT, 1001, 0.05)
        assert_parity(c, reads, offsets, 31, True, "forced overflow k31")
        assert c.stats()["n_overflow_fine"] > 0
        reads, offsets, _ = synth.generate(synth.LONG_NOISY, 1003, 0.002)
        assert_parity(c, reads, offsets, 63, True, "forced overflow k63")
        r, o = as_reads(["T" * 100, "ACGT" * 30, "T" * 32, "GATTACA" * 20])
        assert_parity(c, r, o, 32, False, "forced overflow all-T")
    finally:
        c.close()


def test_deferred_write_out_forced(torch_cuda):
    # every fine partition writes its run to its own input region and the compaction pass
    # moves it to its place (the path of a partition whose output offset was not yet known)
    from paper_2505_04431_gb300 import KmerCounter
    c = KmerCounter(defer_all=True)
    try:
        reads, offsets, _ = synth.generate(synth.REPEAT_SHORT, 1002, 0.003)
        assert_parity(c, reads, offsets, 31, True, "deferred k31")
        st = c.stats()
        assert st["n_deferred_fine"] == st["n_fine"] - st["n_overflow_fine"] > 0
        reads, offsets, _ = synth.generate(synth.LONG_NOISY, 1003, 0.002)
        assert_parity(c, reads, offsets, 63, True, "deferred k63")
        for k in (32, 64):  # the all-ones key, written last in its run
            r, o = as_reads(["T" * 100, "ACGT" * 30, "T" * k, "GGT" + "T" * 70])
            assert_parity(c, r, o, k, False, f"deferred all-T k={k}")
    finally:
        c.close()
    # with tiny tables too: overflowing partitions (which wait for their offset) among
    # deferred ones (which never publish an inclusive prefix)
    c = KmerCounter(defer_all=True, table_slots_max=64)
    try:
        reads, offsets, _ = synth.generate(synth.UNIFORM_SHORT, 1001, 0.02)
        assert_parity(c, reads, offsets, 31, True, "deferred + overflow k31")
        st = c.stats()
        assert st["n_overflow_fine"] > 0 and st["n_deferred_fine"] > 0
    finally:
        c.close()


@pytest.mark.parametrize("hint", [1, 4096])
def test_partition_count_extremes(torch_cuda, hint):
    from paper_2505_04431_gb300 import KmerCounter
    c = KmerCounter(n_partitions_hint=hint)
    try:
        reads, offsets, _ = synth.generate(synth.UNIFORM_SHORT, 1001, 0.2)
        assert_parity(c, reads, offsets, 31, True, f"P1={hint}")
        reads, offsets, _ = synth.generate(synth.LONG_NOISY, 1003, 0.002)
        assert_parity(c, reads, offsets, 63, True, f"P1={hint} k63")
    finally:
        c.close()


def test_input_memory_kinds(counter, torch_cuda):
    torch = torch_cuda
    reads, offsets, _ = synth.generate(synth.UNIFORM_SHORT, 1001, 0.05)
    ok, oc, onv = oracle.count(reads, offsets, 31, True)

    def check(r, o, tag):
        gk, gc, gnv = gpu_count(counter, r, o, 31, True)
        assert gnv == onv and np.array_equal(gk, ok) and np.array_equal(gc, oc), tag

    rt, ot = torch.from_numpy(reads), torch.from_numpy(offsets.astype(np.int64))
    check(reads, offsets, "numpy host")
    check(rt.pin_memory(), ot.pin_memory(), "pinned host")
    check(rt.cuda(), ot.cuda(), "device")
    # device reads at an address that is not 16-byte aligned
    buf = torch.empty(len(reads) + 1, dtype=torch.uint8, device="cuda")
    buf[1:] = rt.cuda()
    check(buf[1:], ot.cuda(), "unaligned device")
    # host offsets, device reads
    check(rt.cuda(), offsets, "mixed")


def test_bad_offsets_rejected(counter, torch_cuda):
    from paper_2505_04431_gb300 import KC_EINVAL, KcError
    reads = np.frombuffer(b"ACGTACGTAC", dtype=np.uint8).copy()
    bad = np.array([0, 6, 3, 10], dtype=np.uint64)
    with pytest.raises(KcError) as e:
        counter.count(reads, bad, 3, True)
    assert e.value.status == KC_EINVAL
    torch = torch_cuda
    with pytest.raises(KcError) as e:
        counter.count(torch.from_numpy(reads).cuda(), torch.from_numpy(bad.astype(np.int64)).cuda(), 3, True)
    assert e.value.status == KC_EINVAL
    with pytest.raises(KcError):
        counter.count(reads, np.array([1, 10], dtype=np.uint64), 3, True)
    for k in (0, 65):
        with pytest.raises(KcError):
            counter.count(reads, np.array([0, 10], dtype=np.uint64), k, True)
    # the plan still works afterwards
    assert_parity(counter, reads, np.array([0, 4, 10], dtype=np.uint64), 3, True, "after errors")


def test_repeated_calls_identical(counter):
    reads, offsets, _ = synth.generate(synth.REPEAT_SHORT, 1002, 0.002)
    a = gpu_count(counter, reads, offsets, 31, True)
    b = gpu_count(counter, reads, offsets, 31, True)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


# ---------------------------------------------------------------- full size, whole histogram
@pytest.mark.parametrize("name", ["repeats_100mbp_150bp_30x_k31", "long_50mbp_10kbp_20x_k63"])
def test_full_size_whole_histogram(counter, torch_cuda, name):
    """Every (key, count) of the full-size workloads, in the configuration bench.py times:
    the SHA-256 of the whole sorted histogram equals the oracle's (stored by
    tests/golden/make_full_size_digests.py, which runs the oracle alone).  If this machine
    generates other reads than the stored input digest says (its math library rounds a
    log-normal read length differently), the oracle counts these reads here instead."""
    import json

    from tests.digest import histogram_digest, input_digest
    from tests.golden.make_full_size_digests import oracle_full_digest
    torch = torch_cuda
    with open(os.path.join(os.path.dirname(__file__), "golden", "full_size_digests.json")) as f:
        golden = json.load(f)[name]
    reads, offsets, k = synth.workload(name)
    if input_digest(reads, offsets) == golden["input_sha256"]:
        want = golden
    else:
        want = oracle_full_digest(reads, offsets, k, True)
    rt = torch.from_numpy(reads).cuda()
    ot = torch.from_numpy(offsets.view(np.int64)).cuda()
    res = counter.count(rt, ot, k, True)
    try:
        assert res.n_valid_windows == want["windows"]
        assert res.n == want["distinct"]
        keys, counts = res.to_numpy()
    finally:
        res.free()
    assert histogram_digest(keys, counts) == want["sha256"]


def test_golden_aatgg_repeat(counter):
    """The paper's heavy-hitter repeat (AATGG)_n, Section IV-D: the GPU path reproduces the
    closed-form histogram of tests/golden/aatgg_repeat.txt."""
    from tests.golden import aatgg_repeat
    reads, offsets, want = aatgg_repeat()
    for (canonical, k), (wk, wc) in want.items():
        res = counter.count(reads, offsets, k, canonical)
        try:
            keys, counts = res.to_numpy()
            assert res.n_valid_windows == reads.size - k + 1
            assert np.array_equal(keys, wk) and np.array_equal(counts, wc), (canonical, k)
        finally:
            res.free()


@pytest.mark.parametrize("no_buckets,merge", [(True, False), (False, True), (True, True)])
def test_aggregation_variants_keep_the_result(torch_cuda, no_buckets, merge):
    """The aggregation variants (pass B without shared-memory buckets, count kernel with the
    warp merge of equal keys) compute the same histogram."""
    from paper_2505_04431_gb300 import KmerCounter
    c = KmerCounter(no_smem_buckets=no_buckets, warp_merge=merge)
    try:
        cases = [synth.generate(synth.REPEAT_SHORT, 1002, 0.001)[:2],
                 (np.frombuffer(b"ACGTTGCA" * 4000, dtype=np.uint8).copy(), np.array([0, 32000], np.uint64))]
        for reads, offsets in cases:
            for k, canonical in ((31, True), (21, False), (63, True)):
                assert_parity(c, reads, offsets, k, canonical, f"variant {no_buckets} {merge} k={k}")
    finally:
        c.close()


# ---------------------------------------------------------------- sampled fine layout
def test_sampled_fine_layout(torch_cuda):
    """Fine partitions' regions sized from a 1/8 sample of the keys (the default for counts of
    2^26 bases and more) forced on medium inputs: the result equals the oracle's."""
    from paper_2505_04431_gb300 import KmerCounter
    c = KmerCounter(test_fine_sampled=True)
    try:
        reads, offsets, _ = synth.generate(synth.REPEAT_SHORT, 1002, 0.03)  # 3 M bases
        assert_parity(c, reads, offsets, 31, True, "sampled k31")
        assert c.stats()["fine_sampled"] == 1
        reads, offsets, _ = synth.generate(synth.LONG_NOISY, 1003, 0.02)  # 20 M bases, 128-bit keys
        assert_parity(c, reads, offsets, 63, True, "sampled k63")
        reads, offsets, _ = synth.generate(synth.UNIFORM_SHORT, 1001, 0.5)
        assert_parity(c, reads, offsets, 21, False, "sampled k21 forward")
    finally:
        c.close()


def test_sampled_layout_overflow_takes_the_exact_split(torch_cuda):
    """Regions without slack overflow: the runs past a region's end are not written, the
    spill is recorded, and the exact fine split that follows gives the oracle's result."""
    from paper_2505_04431_gb300 import KmerCounter
    for extra in ({}, {"defer_all": True}):
        c = KmerCounter(test_fine_sampled=True, test_tight_slack=True, **extra)
        try:
            reads, offsets, _ = synth.generate(synth.REPEAT_SHORT, 1002, 0.03)
            assert_parity(c, reads, offsets, 31, True, f"tight k31 {extra}")
            st = c.stats()
            assert st["fine_sampled"] == 1 and st["fine_resplit"] == 1
            reads, offsets, _ = synth.generate(synth.LONG_NOISY, 1003, 0.02)
            assert_parity(c, reads, offsets, 63, True, f"tight k63 {extra}")
            assert c.stats()["fine_resplit"] == 1
        finally:
            c.close()

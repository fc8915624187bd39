"""The error reports of the C ABI (include/kc.h), each made to happen without a GPU fault:
an allocator that returns NULL, a device-memory limit below what the input needs, a
device-side wait whose limit runs out (partition 0 withholds its prefix under a test-only
plan flag, so the bounded look-back of its successors gives up and returns), and a count
above the reporting limit (a test-only plan flag lowers it to 2^16 - 1, so that the
overflow report is reached without 2^32 windows of one k-mer).  After each failure the
context stays usable: the same input then counts correctly on a normal plan."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_04431_gb300 import build, load_library
    build.build()
    return load_library()


def counts_like_the_oracle(reads, offsets, k):
    from paper_2505_04431_gb300 import KmerCounter
    c = KmerCounter()
    try:
        res = c.count(reads, offsets, k, True)
        keys, counts = res.to_numpy()
        res.free()
    finally:
        c.close()
    ok, oc, _ = oracle.count(reads, offsets, k, True)
    return np.array_equal(keys, ok) and np.array_equal(counts, oc)


def test_allocator_returning_null_gives_enomem(lib):
    from paper_2505_04431_gb300 import _ALLOC_FN, _FREE_FN, KC_ENOMEM, KC_OK, PlanOpts, Result
    reads, offsets, _ = synth.generate(synth.UNIFORM_SHORT, 1001, 0.02)
    calls = []
    alloc = _ALLOC_FN(lambda n, s, c: calls.append(n) or None)
    free = _FREE_FN(lambda p, s, c: None)
    opts = PlanOpts()
    opts.device = 0
    opts.alloc = alloc
    opts.free_ = free
    plan = ctypes.c_void_p()
    assert lib.kc_plan(ctypes.byref(opts), ctypes.byref(plan)) == KC_OK
    try:
        res = Result()
        st = lib.kc_count(plan, reads.ctypes.data, offsets.ctypes.data, len(offsets) - 1, 31, 1, ctypes.byref(res))
        assert st == KC_ENOMEM, lib.kc_last_error()
        assert b"allocation failed" in lib.kc_last_error()
        assert calls and res.n == 0 and not res.keys
    finally:
        lib.kc_plan_destroy(plan)
    assert counts_like_the_oracle(reads, offsets, 31)


def test_device_memory_limit_gives_enomem(lib):
    from paper_2505_04431_gb300 import KC_ENOMEM, KcError, KmerCounter
    reads, offsets, _ = synth.generate(synth.UNIFORM_SHORT, 1001, 0.05)
    c = KmerCounter(max_device_bytes=1 << 20)  # far below the scratch of 5 M bases
    try:
        with pytest.raises(KcError) as e:
            c.count(reads, offsets, 31, True)
        assert e.value.status == KC_ENOMEM and "max_device_bytes" in str(e.value)
        with pytest.raises(KcError) as e:
            c.count_batch([(reads, offsets)] * 2, 31, True)
        assert e.value.status == KC_ENOMEM
        with pytest.raises(KcError) as e:
            c.submit(reads, offsets, 31, True)
        assert e.value.status == KC_ENOMEM
    finally:
        c.close()
    assert counts_like_the_oracle(reads, offsets, 31)


def test_bounded_wait_running_out_gives_etimeout(lib):
    from paper_2505_04431_gb300 import KC_ETIMEOUT, KcError, KmerCounter
    reads, offsets, _ = synth.generate(synth.UNIFORM_SHORT, 1001, 0.2)  # ~150 fine partitions
    c = KmerCounter(test_withhold_prefix=True)
    try:
        for k in (31, 63):
            with pytest.raises(KcError) as e:
                c.count(reads, offsets, k, True)
            assert e.value.status == KC_ETIMEOUT, str(e.value)
            assert c.stats()["n_fine"] >= 2
    finally:
        c.close()
    assert counts_like_the_oracle(reads, offsets, 31)
    assert counts_like_the_oracle(reads, offsets, 63)


def test_count_above_the_limit_gives_eoverflow(lib):
    from paper_2505_04431_gb300 import KC_EOVERFLOW, KcError, KmerCounter

    def homopolymer(n):  # n reads of 150 A's: the k-mer A...A occurs 120 n times (k = 31)
        reads = np.frombuffer(b"A" * 150 * n, dtype=np.uint8).copy()
        return reads, np.arange(n + 1, dtype=np.uint64) * 150

    c = KmerCounter(test_count_limit=True)
    try:
        r, o = homopolymer(546)  # 65520 occurrences: at the limit of 2^16 - 1, reported
        res = c.count(r, o, 31, True)
        keys, counts = res.to_numpy()
        res.free()
        assert keys.tolist() == [0] and counts.tolist() == [65520]
        r, o = homopolymer(547)  # 65640 occurrences: above it
        with pytest.raises(KcError) as e:
            c.count(r, o, 31, True)
        assert e.value.status == KC_EOVERFLOW and "limit" in str(e.value)
    finally:
        c.close()
    assert counts_like_the_oracle(r, o, 31)

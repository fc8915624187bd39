"""Pipelined counts of host inputs: kc_submit copies host reads and offsets in on the plan's
transfer stream, kc_job_copy_to_host has the result copied out there as soon as the count
ends, so that both copies overlap the counts queued around them.  Every result that
arrives in host memory must equal the same input counted alone (kc_count), byte for byte,
and on small inputs the oracle."""
import time

import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


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


def alone(counter, reads, offsets, k, canonical=True):
    res = counter.count(reads, offsets, k, canonical)
    try:
        keys, counts = res.to_numpy()
        return keys, counts, res.n, res.n_valid_windows
    finally:
        res.free()


def host_out(torch, n_windows, k):
    kw = 1 if k <= 32 else 2
    cap = max(1, n_windows)
    return (torch.full((cap * kw,), -1, dtype=torch.int64).pin_memory(),
            torch.full((cap,), -1, dtype=torch.int32).pin_memory())


def test_pipelined_host_counts_equal_counts_alone(counter, torch_cuda):
    """Eight host inputs (pinned and pageable, k = 21, 31, 63, one empty) submitted two
    ahead of collection, each result copied to its own host buffers on the transfer stream."""
    torch = torch_cuda
    inputs = []
    for i in range(7):
        r, o, _ = synth.generate(synth.SERVE, synth.mix_seed(1006, i), 0.02)
        inputs.append((r, o))
    inputs.insert(3, (np.zeros(0, np.uint8), np.zeros(1, np.uint64)))
    ks = [31, 63, 21, 31, 63, 31, 21, 63]
    outs, jobs, results = {}, {}, {}

    def collect(i, by_poll):
        if by_poll:
            t_end = time.time() + 60
            while (res := counter.poll(jobs[i])) is None:
                assert time.time() < t_end
                time.sleep(1e-3)
        else:
            res = counter.wait(jobs[i])
        results[i] = (res.n, res.n_valid_windows)
        res.free()

    for i, ((r, o), k) in enumerate(zip(inputs, ks)):
        if i % 2:  # pinned host memory
            rr, oo = torch.from_numpy(r).pin_memory(), torch.from_numpy(o.view(np.int64)).pin_memory()
        else:  # pageable numpy arrays
            rr, oo = r, o
        jobs[i] = counter.submit(rr, oo, ks[i], True, n_bases=int(o[-1]))
        outs[i] = host_out(torch, max(1, len(r)), k)
        counter.copy_to_host(jobs[i], *outs[i])
        if i >= 2:
            collect(i - 2, by_poll=bool(i % 2))
    for i in range(len(inputs) - 2, len(inputs)):
        collect(i, by_poll=False)
    for i, ((r, o), k) in enumerate(zip(inputs, ks)):
        n, nv = results[i]
        ak, ac, an, anv = alone(counter, r, o, k)
        kw = 1 if k <= 32 else 2
        keys = outs[i][0][: n * kw].numpy().view(np.uint64)
        counts = outs[i][1][:n].numpy().view(np.uint32)
        assert n == an and nv == anv, f"input {i}"
        assert np.array_equal(keys, ak.reshape(-1)) and np.array_equal(counts, ac), f"input {i} differs"
        assert np.all(outs[i][1][n:n + 1].numpy() == -1), "written past the result"
        if i in (0, 3):
            ek, ec, env = oracle.count(r, o, k, True)
            assert env == nv and np.array_equal(keys, ek.reshape(-1)) and np.array_equal(counts, ec)


def test_host_buffers_too_small_fail_the_job_then_counting_goes_on(counter, torch_cuda):
    torch = torch_cuda
    from paper_2505_04431_gb300 import KC_EINVAL, KcError
    r, o, _ = synth.generate(synth.SERVE, synth.mix_seed(1006, 11), 0.01)
    ak, ac, an, _ = alone(counter, r, o, 31)
    job = counter.submit(r, o, 31, True, n_bases=int(o[-1]))
    small = (torch.zeros(an - 1, dtype=torch.int64).pin_memory(), torch.zeros(an - 1, dtype=torch.int32).pin_memory())
    counter.copy_to_host(job, *small)
    with pytest.raises(KcError) as e:
        counter.wait(job)
    assert e.value.status == KC_EINVAL and "does not fit" in str(e.value)
    with pytest.raises(KcError) as e:  # the job is gone
        counter.copy_to_host(job, *small)
    assert e.value.status == KC_EINVAL
    # the plan counts on
    job = counter.submit(r, o, 31, True, n_bases=int(o[-1]))
    out = host_out(torch, an, 31)
    counter.copy_to_host(job, *out)
    res = counter.wait(job)
    assert res.n == an
    res.free()
    assert np.array_equal(out[0][:an].numpy().view(np.uint64), ak) and np.array_equal(out[1][:an].numpy().view(np.uint32), ac)


def test_unordered_host_offsets_are_reported_when_collected(counter, torch_cuda):
    """Host offsets are checked for order on the device (only their ends on the host)."""
    from paper_2505_04431_gb300 import KC_EINVAL, KcError
    r, o, _ = synth.generate(synth.SERVE, synth.mix_seed(1006, 12), 0.01)
    bad = o.copy()
    bad[5], bad[6] = bad[6], bad[5]  # decreasing between reads 4 and 6
    assert bad[6] < bad[5]
    job = counter.submit(r, bad, 31, True, n_bases=int(o[-1]))
    with pytest.raises(KcError) as e:
        counter.wait(job)
    assert e.value.status == KC_EINVAL
    ak, ac, an, _ = alone(counter, r, o, 31)
    job = counter.submit(r, o, 31, True, n_bases=int(o[-1]))
    res = counter.wait(job)
    keys, counts = res.to_numpy()
    res.free()
    assert np.array_equal(keys, ak) and np.array_equal(counts, ac)


@pytest.mark.parametrize("tight", [False, True])
def test_pipelined_counts_with_sampled_fine_layouts(counter, torch_cuda, tight):
    """Submitted host counts on a plan that sizes fine partition regions from a sample at
    every size (with `tight`, with no slack, so that regions spill and the exact fine split
    runs inside the job): every result copied out equals the plain plan's count alone."""
    torch = torch_cuda
    from paper_2505_04431_gb300 import KmerCounter
    c = KmerCounter(test_fine_sampled=True, test_tight_slack=tight)
    try:
        inputs = [synth.generate(synth.REPEAT_SHORT, 1002, 0.03)[:2],  # 3 M bases
                  synth.generate(synth.LONG_NOISY, 1003, 0.02)[:2],  # 20 M bases, 128-bit keys
                  synth.generate(synth.SERVE, synth.mix_seed(1007, 0), 0.03)[:2],
                  synth.generate(synth.SERVE, synth.mix_seed(1007, 1), 0.03)[:2]]
        ks = [31, 63, 21, 31]
        jobs, outs, got = [], [], []
        for (r, o), k in zip(inputs, ks):
            j = c.submit(r, o, k, True, n_bases=int(o[-1]))
            out = host_out(torch, max(1, len(r)), k)
            c.copy_to_host(j, *out)
            jobs.append(j)
            outs.append(out)
        resplit = 0
        for j in jobs:
            res = c.wait(j)
            got.append((res.n, res.n_valid_windows))
            resplit += c.stats()["fine_resplit"]
            res.free()
        for i, ((r, o), k) in enumerate(zip(inputs, ks)):
            ak, ac, an, anv = alone(counter, r, o, k)
            n, nv = got[i]
            kw = 1 if k <= 32 else 2
            assert n == an and nv == anv, f"input {i}"
            assert np.array_equal(outs[i][0][: n * kw].numpy().view(np.uint64), ak.reshape(-1)), f"input {i} keys"
            assert np.array_equal(outs[i][1][:n].numpy().view(np.uint32), ac), f"input {i} counts"
        if tight:
            assert resplit > 0, "no region spilled with tight slack"
    finally:
        c.close()


def test_copy_to_host_checks_the_buffers_against_the_job(counter, torch_cuda):
    """The binding refuses host buffers whose element sizes, or whose key words for the job's
    k, do not fit, before the C call takes their plain pointers; the job is then collected
    as usual."""
    torch = torch_cuda
    r, o, _ = synth.generate(synth.SERVE, synth.mix_seed(1006, 13), 0.01)
    cap = max(1, len(r))
    job = counter.submit(r, o, 63, True, n_bases=int(o[-1]))
    with pytest.raises(ValueError):  # one word per key, where k = 63 keys take two
        counter.copy_to_host(job, torch.empty(cap, dtype=torch.int64), torch.empty(cap, dtype=torch.int32))
    with pytest.raises(ValueError):  # 64-bit counts
        counter.copy_to_host(job, torch.empty(2 * cap, dtype=torch.int64), torch.empty(cap, dtype=torch.int64))
    res = counter.wait(job)
    keys, counts = res.to_numpy()
    n = res.n
    res.free()
    ak, ac, an, _ = alone(counter, r, o, 63)
    assert n == an and np.array_equal(keys, ak) and np.array_equal(counts, ac)

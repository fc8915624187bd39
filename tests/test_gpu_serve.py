"""Submitted counts (kc_submit / kc_job_poll / kc_job_wait) and the served forms on the
GPU: every result is byte-identical to the same input counted alone (kc_count), and on
small inputs to the oracle."""
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
        return keys, counts, res.n_valid_windows
    finally:
        res.free()


def test_submitted_counts_match_single_counts(counter, torch_cuda):
    torch = torch_cuda
    inputs = []
    for i in range(10):  # genomes of 1 kbp - 0.4 Mbp at 10-30x, all queued before any is collected
        r, o, _ = synth.generate(synth.SERVE, synth.mix_seed(1005, i), 0.02)
        inputs.append((r, o))
    inputs.insert(4, (np.zeros(0, np.uint8), np.zeros(1, np.uint64)))  # an empty input
    ks = [21, 31, 63, 31, 21, 63, 31, 31, 21, 63, 31]
    jobs = []
    for i, ((r, o), k) in enumerate(zip(inputs, ks)):
        if i % 2:  # pinned host reads and offsets
            rr = torch.from_numpy(r).pin_memory()
            oo = torch.from_numpy(o.view(np.int64)).pin_memory()
        else:  # device reads and offsets
            rr = torch.from_numpy(r).cuda()
            oo = torch.from_numpy(o.view(np.int64)).cuda()
        torch.cuda.synchronize()
        jobs.append(counter.submit(rr, oo, k, True, n_bases=int(o[-1])))
    assert len(set(jobs)) == len(jobs) and all(j > 0 for j in jobs)
    results = {}
    for i in reversed(range(len(jobs))):  # collect out of submission order, by wait and by poll
        if i % 3 == 0:
            results[i] = counter.wait(jobs[i])
        else:
            t_end = time.time() + 60
            while (res := counter.poll(jobs[i])) is None:
                assert time.time() < t_end
                time.sleep(1e-3)
            results[i] = res
    for i, ((r, o), k) in enumerate(zip(inputs, ks)):
        res = results[i]
        keys, counts = res.to_numpy()
        nv = res.n_valid_windows
        res.free()
        ak, ac, anv = alone(counter, r, o, k)
        assert nv == anv and np.array_equal(keys, ak) and np.array_equal(counts, ac), f"input {i} differs"
        if i in (0, 4):
            ek, ec, env = oracle.count(r, o, k, True)
            assert env == nv and np.array_equal(keys, ek) and np.array_equal(counts, ec)


def test_submit_errors_and_recovery(counter, torch_cuda):
    from paper_2505_04431_gb300 import KC_EINVAL, KcError
    torch = torch_cuda
    reads = np.frombuffer(b"ACGTACGTAC", dtype=np.uint8).copy()
    bad = np.array([0, 6, 3, 10], dtype=np.uint64)
    with pytest.raises(KcError) as e:  # host offsets whose ends are wrong: refused at once, no job
        counter.submit(reads, np.array([0, 10], np.uint64), 3, True, n_bases=9)
    assert e.value.status == KC_EINVAL
    with pytest.raises(KcError) as e:
        counter.submit(reads, np.array([1, 10], np.uint64), 3, True, n_bases=10)
    assert e.value.status == KC_EINVAL
    # host offsets out of order: their order is checked on the GPU, reported when collected
    job = counter.submit(reads, bad, 3, True, n_bases=10)
    with pytest.raises(KcError) as e:
        counter.wait(job)
    assert e.value.status == KC_EINVAL
    # device offsets: the GPU finds the error; it is reported when the job is collected
    job = counter.submit(torch.from_numpy(reads).cuda(), torch.from_numpy(bad.astype(np.int64)).cuda(), 3, True,
                         n_bases=10)
    with pytest.raises(KcError) as e:
        counter.wait(job)
    assert e.value.status == KC_EINVAL
    with pytest.raises(KcError) as e:  # the job id is gone
        counter.poll(job)
    assert e.value.status == KC_EINVAL
    # the plan still counts correctly
    o = np.array([0, 4, 10], dtype=np.uint64)
    res = counter.wait(counter.submit(reads, o, 3, True))
    keys, counts = res.to_numpy()
    res.free()
    ek, ec, _ = oracle.count(reads, o, 3, True)
    assert np.array_equal(keys, ek) and np.array_equal(counts, ec)


def test_uncollected_jobs_released_on_close(torch_cuda):
    from paper_2505_04431_gb300 import KmerCounter
    torch = torch_cuda
    c = KmerCounter()
    r, o, _ = synth.generate(synth.SERVE, synth.mix_seed(1005, 1), 0.01)
    rd = torch.from_numpy(r).cuda()
    torch.cuda.synchronize()
    for k in (21, 31, 63):
        c.submit(rd, o, k, True)
    c.close()  # waits for the three and frees their buffers
    torch.cuda.synchronize()


def make_requests(torch, n=40, seed=7):
    """n requests over 6 read sets: the first half arrive at once (so that requests surely
    wait together), the rest at Poisson times."""
    from paper_2505_04431_gb300 import serve as sv
    pool = []
    for i in range(6):
        r, o, _ = synth.generate(synth.SERVE, synth.mix_seed(1005, i), 0.02)
        pool.append((torch.from_numpy(r).cuda(), torch.from_numpy(o.view(np.int64)).cuda(), int(o[-1])))
    torch.cuda.synchronize()
    rng = np.random.RandomState(seed)
    arrivals = np.cumsum(rng.exponential(0.002, n))
    arrivals[: n // 2] = 0.0
    return [sv.Request(float(t), *pool[p], int(k)) for t, p, k in
            zip(arrivals, rng.randint(0, 6, n), rng.choice([21, 31, 63], n))]


def digests_alone(counter, reqs):
    from paper_2505_04431_gb300 import serve as sv
    out = []
    for r in reqs:
        res = counter.count(r.reads, r.offsets, r.k)
        try:
            out.append(sv.result_digest(res))
        finally:
            res.free()
    return out


def test_served_async_results_identical_to_single_counts(counter, torch_cuda):
    from paper_2505_04431_gb300 import serve as sv
    reqs = make_requests(torch_cuda)
    info = sv.serve_async(counter, reqs, budget_bytes=2 << 30, on_result=lambda r, res: res.free())
    assert info["peak_inflight"] > 1  # requests were queued behind each other
    assert [r.digest for r in reqs] == digests_alone(counter, reqs)
    assert all(r.done >= r.arrival for r in reqs)


def test_served_batches_identical_to_single_counts(counter, torch_cuda):
    from paper_2505_04431_gb300 import serve as sv
    reqs = make_requests(torch_cuda, seed=8)
    info = sv.serve(counter, reqs, budget_bytes=2 << 30, on_result=lambda r, res: res.free())
    assert info["batches"] < len(reqs)  # requests were batched
    assert [r.digest for r in reqs] == digests_alone(counter, reqs)


def test_submit_batch_matches_single_counts(counter, torch_cuda):
    # a 32 MiB arena: several groups of batched launches and counts alone in one submission;
    # two submissions queued before anything is collected, collected out of order
    from paper_2505_04431_gb300 import KC_EINVAL, KcError, KmerCounter
    torch = torch_cuda
    inputs = []
    for i in range(9):
        r, o, _ = synth.generate(synth.SERVE, synth.mix_seed(3005, i), 0.02)
        inputs.append((r, o))
    inputs.insert(2, (np.zeros(0, np.uint8), np.zeros(1, np.uint64)))
    small = KmerCounter(small_batch_arena=True)
    try:
        dev = [(torch.from_numpy(r).cuda(), torch.from_numpy(o.view(np.int64)).cuda(), int(o[-1])) for r, o in inputs]
        torch.cuda.synchronize()
        with pytest.raises(KcError) as e:  # bad host offsets: refused, no job
            bad = inputs[0][1].copy()
            bad[1], bad[2] = bad[2], bad[1]
            small.submit_batch([dev[1], (dev[0][0], bad, int(bad[-1]))], 31)
        assert e.value.status == KC_EINVAL
        jobs31 = small.submit_batch(dev[:6], 31)
        jobs63 = small.submit_batch(dev[4:], 63)
        want = [(i, 31, j) for i, j in enumerate(jobs31)] + [(4 + i, 63, j) for i, j in enumerate(jobs63)]
        got = {}
        for i, k, j in reversed(want):
            if j % 2:
                got[j] = small.wait(j)
            else:
                t_end = time.time() + 60
                while (res := small.poll(j)) is None:
                    assert time.time() < t_end
                    time.sleep(1e-3)
                got[j] = res
        for i, k, j in want:
            res = got[j]
            keys, counts = res.to_numpy()
            nv = res.n_valid_windows
            r, o = inputs[i]
            ak, ac, anv = alone(counter, r, o, k)
            assert nv == anv and np.array_equal(keys, ak) and np.array_equal(counts, ac), f"input {i}, k {k}"
        for j in np.random.RandomState(3).permutation([j for _, _, j in want]):
            got[int(j)].free()
    finally:
        small.close()


def test_served_async_batched_identical_to_single_counts(counter, torch_cuda):
    from paper_2505_04431_gb300 import serve as sv
    reqs = make_requests(torch_cuda, n=60, seed=9)
    info = sv.serve_async(counter, reqs, budget_bytes=2 << 30, policy="sjf", batch=True,
                          on_result=lambda r, res: res.free())
    assert info["batches"] < len(reqs)  # some requests shared a submission
    assert [r.digest for r in reqs] == digests_alone(counter, reqs)

"""Host logic of the served form (no GPU): admission by free device memory and under an
optional budget, one kc_count_batch call per k and round, arrival order, results handed to
the caller, latency summary."""
import numpy as np
import pytest

from paper_2505_04431_gb300 import serve as sv


class FakeResult:
    def __init__(self, n):
        self.n = n
        self.n_valid_windows = n

    def free(self):
        pass


def fake_footprint(n_reads, n_bases, k, reads_on_device=True, offsets_on_device=True):
    return 16 * n_bases, 12 * n_bases  # (scratch, result)


def plenty():
    return 1 << 60


class FakeCounter:
    """Records the calls; a 'count' takes no time."""

    def __init__(self):
        self.batches = []
        self.singles = []

    footprint = staticmethod(fake_footprint)

    def count_batch(self, samples, k, canonical=True):
        self.batches.append((k, [s[2] for s in samples]))
        return [FakeResult(s[2]) for s in samples]

    def count(self, reads, offsets, k, canonical=True):
        self.singles.append((k, int(offsets[-1])))
        return FakeResult(int(offsets[-1]))


def req(t, n, k):
    return sv.Request(t, None, np.array([0, n], np.uint64), n, k)


def test_all_arrived_requests_are_batched_by_k():
    c = FakeCounter()
    reqs = [req(0.0, 100, 21), req(0.0, 200, 31), req(0.0, 300, 21), req(0.0, 400, 63)]
    info = sv.serve(c, reqs, budget_bytes=1 << 40, mem_free=plenty, keep_digest=False)
    assert sorted(c.batches) == [(21, [100, 300]), (31, [200]), (63, [400])]
    assert info["batches"] == 3
    assert all(r.done >= r.arrival and r.n_distinct == r.n_bases for r in reqs)


def test_budget_limits_a_round_but_admits_at_least_one():
    c = FakeCounter()
    big = 1 << 30
    reqs = [req(0.0, big, 31), req(0.0, big, 31), req(0.0, 10, 31)]
    budget = sv.footprint(c, reqs[0]) + sv.footprint(c, reqs[2])  # the second big one does not fit with the first
    sv.serve(c, reqs, budget_bytes=budget, mem_free=plenty, keep_digest=False)
    assert c.batches[0] == (31, [big, 10])  # arrival order, skipping what does not fit
    assert c.batches[1] == (31, [big])
    c2 = FakeCounter()
    sv.serve(c2, [req(0.0, big, 31)], budget_bytes=1, mem_free=plenty, keep_digest=False)  # alone above the budget: still served
    assert c2.batches == [(31, [big])]


def test_requests_wait_for_their_arrival_and_plain_loop_is_fifo():
    c = FakeCounter()
    reqs = [req(0.03, 5, 21), req(0.0, 7, 31)]
    sv.serve(c, reqs, budget_bytes=1 << 40, mem_free=plenty, keep_digest=False)
    assert c.batches[0] == (31, [7])  # the later arrival is not counted before it arrives
    assert reqs[0].done >= 0.03
    c2 = FakeCounter()
    sv.serve_one_at_a_time(c2, [req(0.02, 5, 21), req(0.0, 7, 31)], keep_digest=False)
    assert c2.singles == [(31, 7), (21, 5)]
    lat = sv.latency_summary(reqs)
    assert lat["p50_ms"] >= 0 and lat["p99_ms"] >= lat["p50_ms"]



class FakeAsyncCounter:
    """submit / poll with jobs that finish a fixed time after submission."""

    def __init__(self, seconds_per_base=0.0):
        self.spb = seconds_per_base
        self.jobs = {}
        self.submitted = []
        self.batches = []
        self.submit_times = []
        self.max_inflight = 0
        self.next = 1

    footprint = staticmethod(fake_footprint)

    def submit(self, reads, offsets, k, canonical=True, n_bases=None):
        import time
        jid = self.next
        self.next += 1
        self.jobs[jid] = (time.perf_counter() + self.spb * n_bases, n_bases)
        self.submitted.append((k, n_bases))
        self.submit_times.append(time.perf_counter())
        self.max_inflight = max(self.max_inflight, len(self.jobs))
        return jid

    def submit_batch(self, samples, k, canonical=True):
        import time
        self.batches.append((k, [sm[2] for sm in samples]))
        t_end = time.perf_counter() + self.spb * sum(sm[2] for sm in samples)
        out = []
        for sm in samples:
            jid = self.next
            self.next += 1
            self.jobs[jid] = (t_end, sm[2])  # a batch completes as a whole
            self.submitted.append((k, sm[2]))
            out.append(jid)
        self.max_inflight = max(self.max_inflight, len(self.jobs))
        return out

    def poll(self, job):
        import time
        t, n = self.jobs[job]
        if time.perf_counter() < t:
            return None
        del self.jobs[job]
        return FakeResult(n)


def test_async_submits_in_arrival_order_and_completes_everything():
    c = FakeAsyncCounter()
    reqs = [req(0.01, 5, 21), req(0.0, 7, 31), req(0.02, 9, 63)]
    info = sv.serve_async(c, reqs, budget_bytes=1 << 40, mem_free=plenty, keep_digest=False)
    assert c.submitted == [(31, 7), (21, 5), (63, 9)]
    assert all(r.done >= r.arrival and r.n_distinct == r.n_bases for r in reqs)
    assert not c.jobs and info["batches"] == 3


def test_async_small_request_is_not_held_behind_a_large_one():
    # the large request takes ~0.2 s; the small one, arriving later, finishes long before it
    c = FakeAsyncCounter(seconds_per_base=0.2 / 1000)
    big, small = req(0.0, 1000, 31), req(0.01, 10, 31)
    sv.serve_async(c, [big, small], budget_bytes=1 << 40, mem_free=plenty, keep_digest=False)
    assert small.done < big.done
    assert small.done - small.arrival < 0.1
    assert c.max_inflight == 2


def test_async_budget_holds_back_what_does_not_fit():
    c = FakeAsyncCounter(seconds_per_base=0.05 / (1 << 30))
    big = 1 << 30
    reqs = [req(0.0, big, 31), req(0.0, big, 31), req(0.0, 10, 31)]
    budget = sv.footprint(c, reqs[0]) + sv.footprint(c, reqs[2])
    sv.serve_async(c, reqs, budget_bytes=budget, mem_free=plenty, keep_digest=False)
    # FIFO: the second big one waits for the first to finish, and the small one behind it
    assert c.submitted == [(31, big), (31, big), (31, 10)]
    t_first_done = c.submit_times[0] + 0.05
    assert min(c.submit_times[1:]) >= t_first_done - 1e-3
    assert reqs[1].done > reqs[0].done and reqs[2].done > reqs[0].done
    c2 = FakeAsyncCounter()
    sv.serve_async(c2, [req(0.0, big, 31)], budget_bytes=1, mem_free=plenty, keep_digest=False)  # alone above the budget
    assert c2.submitted == [(31, big)]


def test_async_sjf_runs_short_requests_first_within_the_depth():
    # a large count (~50 ms) occupies the GPU; meanwhile a second large one and three small
    # ones arrive: the small ones go next, the large one after them
    c = FakeAsyncCounter(seconds_per_base=0.05 / 10**9)
    big, small = 10**9, [10**5, 2 * 10**5, 5 * 10**4]
    reqs = [req(0.0, big, 31), req(0.005, big, 31)] + [req(0.006 + 0.001 * i, n, 31) for i, n in enumerate(small)]
    sv.serve_async(c, reqs, budget_bytes=1 << 50, mem_free=plenty, keep_digest=False, policy="sjf", depth=1)
    assert c.max_inflight == 1
    assert c.submitted[0] == (31, big) and c.submitted[-1] == (31, big)
    assert sorted(n for _, n in c.submitted[1:4]) == sorted(small)
    assert reqs[1].done > max(r.done for r in reqs[2:])


def test_async_sjf_ageing_lets_a_long_waiting_request_through():
    c = FakeAsyncCounter()
    long_wait = req(0.0, 10**9, 31)  # expected to take ~40 ms, but it has waited 1 s
    fresh = req(1.0, 10, 31)
    waiting_since = 1.0
    assert sv.expected_seconds(long_wait) - waiting_since < sv.expected_seconds(fresh) - 0.0
    with pytest.raises(ValueError):
        sv.serve_async(c, [fresh], budget_bytes=1, mem_free=plenty, keep_digest=False, policy="lifo")


def test_async_batching_groups_waiting_requests_of_one_k():
    # a long count occupies the GPU (depth 1); meanwhile small requests of two k values
    # arrive; they go in one batched submission per k, the k = 63 ones apart, and one
    # request far larger than the others stays out of their batch
    c = FakeAsyncCounter(seconds_per_base=0.05 / 10**9)
    first = req(0.0, 10**9, 31)
    small31 = [req(0.002 + 0.001 * i, 10**5 * (i + 1), 31) for i in range(4)]
    small63 = [req(0.003 + 0.001 * i, 10**5, 63) for i in range(3)]
    huge31 = req(0.004, 10**9, 31)
    reqs = [first] + small31 + small63 + [huge31]
    info = sv.serve_async(c, reqs, budget_bytes=1 << 50, mem_free=plenty, keep_digest=False, policy="sjf", depth=1, batch=True)
    assert [k for k, _ in c.batches] == [31, 63] or [k for k, _ in c.batches] == [63, 31]
    b31 = dict(c.batches)[31]
    assert sorted(b31) == sorted(r.n_bases for r in small31)  # the huge one is not in it
    assert sorted(dict(c.batches)[63]) == [10**5] * 3
    assert info["batches"] == 4  # first, two batches, huge
    assert all(r.done >= r.arrival and r.n_distinct == r.n_bases for r in reqs)
    assert huge31.done > max(r.done for r in small31 + small63)


def test_async_batching_respects_budget_and_max_batch():
    c = FakeAsyncCounter(seconds_per_base=0.05 / 10**9)
    blocker = req(0.0, 10**9, 21)
    many = [req(0.001, 10**5, 21) for _ in range(10)]
    budget = sv.footprint(c, blocker) + 3 * sv.footprint(c, many[0])
    sv.serve_async(c, [blocker] + many, budget_bytes=budget, mem_free=plenty, keep_digest=False, policy="fifo", depth=1, batch=True,
                   max_batch=6)
    sizes = [len(b) for _, b in c.batches]
    assert max(sizes) <= 6 and sum(sizes) + (len(c.submitted) - sum(sizes)) == 11
    assert all(r.done >= r.arrival for r in many)


def test_admission_follows_free_device_memory():
    # the device has room for one big request and a small one: the second big one waits
    # until the first has finished (FIFO, so the small one waits behind it); every result
    # goes to the caller's on_result, none is kept by the server
    c = FakeAsyncCounter(seconds_per_base=0.05 / (1 << 30))
    big = 1 << 30
    reqs = [req(0.0, big, 31), req(0.0, big, 31), req(0.0, 10, 31)]
    cap = sv.footprint(c, reqs[0]) + sv.footprint(c, reqs[2])

    def mem_free():  # what the jobs in flight leave free
        return cap - sum(28 * n for _, n in c.jobs.values())

    held = []
    sv.serve_async(c, reqs, keep_digest=False, mem_free=mem_free, headroom=0,
                   on_result=lambda r, res: held.append(res))
    assert c.submitted == [(31, big), (31, big), (31, 10)]
    assert min(c.submit_times[1:]) >= c.submit_times[0] + 0.05 - 1e-3
    assert len(held) == 3 and all(r.result is None for r in reqs)


def test_results_stay_with_the_request_by_default():
    c = FakeCounter()
    reqs = [req(0.0, 100, 21), req(0.0, 200, 31)]
    sv.serve(c, reqs, keep_digest=False, mem_free=plenty)
    assert [r.result.n for r in reqs] == [100, 200]
    c2 = FakeCounter()
    reqs2 = [req(0.0, 7, 31)]
    sv.serve_one_at_a_time(c2, reqs2, keep_digest=False)
    assert reqs2[0].result.n == 7

"""Served form: request loops over the k-mer counter.

Count requests (a read set and k) arrive over time; each request's latency runs from its
arrival to the moment its result is complete on the device.  Servers:

- serve_async (the served form): arrived requests are admitted while the device's free
  memory covers what they take (kc_footprint: their result buffers and the scratch they
  need), submitted at once (kc_submit) and queued on the plan's stream; results are
  collected as they complete (kc_job_poll), so the GPU runs the requests back to back
  with no host round trip between them, and the host prepares and checks requests while
  the GPU counts.  With continuous batching, waiting requests of one k go together in one
  submission of batched launches (kc_submit_batch): their thread blocks share every
  kernel launch, so their work overlaps on the device.
- serve: rounds of kc_count_batch over the requests that arrived meanwhile (one call per
  k), for bursts of many requests.
- serve_one_at_a_time: the plain loop, one kc_count per request.

Every server hands each result to on_result(request, result) as soon as it is complete;
by default the result stays on the device in request.result until the caller frees it
(result.free()).  No part of the counting happens here: this module only orders calls
into the library.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np


@dataclasses.dataclass
class Request:
    arrival: float     # seconds after the start of the run
    reads: object      # ASCII bases: a device tensor, or pinned host memory
    offsets: object    # n_reads + 1 offsets: device tensor, or host (pinned for serve_async)
    n_bases: int
    k: int
    done: float = -1.0
    n_distinct: int = -1
    n_valid: int = -1
    digest: tuple = ()
    result: object = None  # the result, kept on the device (default on_result)


def _on_device(x) -> bool:
    return bool(getattr(x, "is_cuda", False))


def footprint(counter, req: Request) -> int:
    """Device bytes the request takes while it is in flight: the scratch its count needs
    and its result buffers (kc_footprint on the counter's plan)."""
    n_reads = (req.offsets.shape[0] if hasattr(req.offsets, "shape") else len(req.offsets)) - 1
    on_dev = _on_device(req.reads) and (req.reads.data_ptr() % 16 == 0)
    scratch, result = counter.footprint(n_reads, req.n_bases, req.k, on_dev, _on_device(req.offsets))
    return scratch + result


def device_free_bytes() -> int:
    """Device memory a count can still get: what the driver reports free, plus what torch's
    caching allocator holds without using it (the library allocates through it)."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    return int(free + torch.cuda.memory_reserved() - torch.cuda.memory_allocated())


def result_digest(res):
    """(distinct keys, valid windows, SHA-256 of the whole sorted result): two results have
    the same digest only if they hold the same keys with the same counts, entry by entry."""
    import hashlib
    keys, counts = res.to_numpy()
    h = hashlib.sha256()
    h.update(keys.tobytes())
    h.update(counts.tobytes())
    return (res.n, res.n_valid_windows, h.hexdigest())


def keep_result(r: Request, res):
    r.result = res


def _finish(r: Request, res, t_done: float, keep_digest: bool, on_result):
    r.done = t_done
    r.n_distinct, r.n_valid = res.n, res.n_valid_windows
    if keep_digest:
        r.digest = result_digest(res)
    (on_result or keep_result)(r, res)


# service time a count is expected to take (ordering only): per base, by key width, plus a
# fixed part for the launches
SECONDS_PER_BASE = {1: 1.0 / 25e9, 2: 1.0 / 12e9}
SECONDS_FIXED = 0.3e-3


def expected_seconds(req: Request) -> float:
    return SECONDS_FIXED + req.n_bases * SECONDS_PER_BASE[1 if req.k <= 32 else 2]


class _Admission:
    """Admits work while free device memory (less `headroom`) covers it, and, with a budget,
    while the footprints in flight stay within it.  One request is always admitted when
    nothing is in flight, whatever it takes."""

    def __init__(self, counter, mem_free, headroom, budget_bytes):
        self.counter = counter
        self.mem_free = mem_free or device_free_bytes
        self.headroom = headroom
        self.budget = budget_bytes
        self.used = 0

    def fits(self, need: int, idle: bool) -> bool:
        if idle:
            return True
        if self.budget is not None and self.used + need > self.budget:
            return False
        return need <= self.mem_free() - self.headroom


def serve_async(counter, requests: list[Request], canonical: bool = True, keep_digest: bool = True,
                idle_sleep: float = 50e-6, policy: str = "fifo", depth: int | None = None, batch: bool = False,
                max_batch: int = 64, batch_ratio: float = 4.0, on_result=None, mem_free=None,
                headroom: int = 1 << 30, budget_bytes: int | None = None):
    """Submit arrived requests while free device memory covers their footprints (and, with
    `depth`, while fewer than `depth` submissions are in flight); collect results as they
    complete.  policy "fifo" takes the waiting requests in arrival order; "sjf" takes next
    the one with the least expected service time minus the time it has waited (shortest
    first, with ageing so that a large request is not held back for ever), and defaults to
    depth 2, so that the GPU always has the next submission queued.  With `batch`
    (continuous batching), the waiting requests with the same k whose expected service time
    is at most `batch_ratio` times that of the request taken (or under 1 ms) join it, in
    policy order and while memory covers them, in one submission of batched launches
    (kc_submit_batch, at most `max_batch` requests).  mem_free() gives the free device
    bytes (default device_free_bytes); budget_bytes optionally caps the footprints in
    flight as well."""
    if policy not in ("fifo", "sjf"):
        raise ValueError(f"unknown policy {policy!r}")
    if depth is None and policy == "sjf":
        depth = 2
    adm = _Admission(counter, mem_free, headroom, budget_bytes)
    queue = collections.deque(sorted(requests, key=lambda r: r.arrival))
    waiting: list = []
    inflight: dict = {}  # job id -> (request, footprint, submission)
    open_subs: dict = {}  # submission -> its jobs still in flight
    next_sub = 0
    peak_inflight = 0
    submissions = 0
    t0 = time.perf_counter()
    while queue or waiting or inflight:
        now = time.perf_counter() - t0
        while queue and queue[0].arrival <= now:
            waiting.append(queue.popleft())
        while waiting and (depth is None or len(open_subs) < depth):
            if policy == "sjf":
                prio = lambda q: expected_seconds(waiting[q]) - (now - waiting[q].arrival)  # noqa: E731
            else:
                prio = lambda q: q  # noqa: E731
            i = min(range(len(waiting)), key=prio)
            r = waiting[i]
            f = footprint(counter, r)
            if not adm.fits(f, not inflight):
                break
            group, need, feet = [i], f, {i: f}
            if batch:
                cap = max(batch_ratio * expected_seconds(r), 1e-3)
                for q in sorted((q for q in range(len(waiting)) if q != i and waiting[q].k == r.k), key=prio):
                    if len(group) >= max_batch:
                        break
                    if expected_seconds(waiting[q]) > cap:
                        continue
                    fq = footprint(counter, waiting[q])
                    if adm.fits(need + fq, False):
                        group.append(q)
                        need += fq
                        feet[q] = fq
            reqs = [waiting[q] for q in group]
            if len(reqs) == 1:
                jobs = [counter.submit(r.reads, r.offsets, r.k, canonical, n_bases=r.n_bases)]
            else:
                jobs = counter.submit_batch([(x.reads, x.offsets, x.n_bases) for x in reqs], r.k, canonical)
            open_subs[next_sub] = len(jobs)
            for job, q in zip(jobs, group):
                inflight[job] = (waiting[q], feet[q], next_sub)
            next_sub += 1
            submissions += 1
            adm.used += need
            for q in sorted(group, reverse=True):
                waiting.pop(q)
        peak_inflight = max(peak_inflight, len(inflight))
        progressed = False
        for job in list(inflight):
            res = counter.poll(job)
            if res is None:
                continue
            r, f, sub = inflight.pop(job)
            adm.used -= f
            open_subs[sub] -= 1
            if not open_subs[sub]:
                del open_subs[sub]
            _finish(r, res, time.perf_counter() - t0, keep_digest, on_result)
            progressed = True
        if not progressed:
            if not inflight and not waiting and queue:
                time.sleep(max(0.0, min(queue[0].arrival - (time.perf_counter() - t0), 0.002)))
            else:
                time.sleep(idle_sleep)
    return {"batches": submissions, "peak_inflight": peak_inflight, "makespan": time.perf_counter() - t0}


def serve(counter, requests: list[Request], canonical: bool = True, keep_digest: bool = True, on_result=None,
          mem_free=None, headroom: int = 1 << 30, budget_bytes: int | None = None):
    """Rounds of kc_count_batch in arrival order: each round takes the arrived requests
    that free device memory covers (at least one), one call per k."""
    adm = _Admission(counter, mem_free, headroom, budget_bytes)
    queue = collections.deque(sorted(requests, key=lambda r: r.arrival))
    waiting: list[Request] = []
    t0 = time.perf_counter()
    batches = 0
    while queue or waiting:
        now = time.perf_counter() - t0
        while queue and queue[0].arrival <= now:
            waiting.append(queue.popleft())
        if not waiting:
            time.sleep(max(0.0, min(queue[0].arrival - now, 0.002)))
            continue
        # admit in arrival order while memory holds (at least one request per round)
        admitted, need = [], 0
        for r in waiting:
            f = footprint(counter, r)
            if admitted and not adm.fits(need + f, False):
                continue
            admitted.append(r)
            need += f
        admitted_ids = {id(r) for r in admitted}
        waiting = [r for r in waiting if id(r) not in admitted_ids]
        by_k = collections.defaultdict(list)
        for r in admitted:
            by_k[r.k].append(r)
        for k, group in sorted(by_k.items()):
            results = counter.count_batch([(r.reads, r.offsets, r.n_bases) for r in group], k, canonical)
            t_done = time.perf_counter() - t0
            for r, res in zip(group, results):
                _finish(r, res, t_done, keep_digest, on_result)
            batches += 1
    return {"batches": batches, "makespan": time.perf_counter() - t0}


def serve_one_at_a_time(counter, requests: list[Request], canonical: bool = True, keep_digest: bool = True,
                        on_result=None):
    """The plain loop: one kc_count per request, first come first served."""
    queue = sorted(requests, key=lambda r: r.arrival)
    t0 = time.perf_counter()
    for r in queue:
        now = time.perf_counter() - t0
        if r.arrival > now:
            time.sleep(r.arrival - now)
        res = counter.count(r.reads, r.offsets, r.k, canonical)
        _finish(r, res, time.perf_counter() - t0, keep_digest, on_result)
    return {"batches": len(queue), "makespan": time.perf_counter() - t0}


def latency_summary(requests: list[Request]) -> dict:
    lat = np.array([r.done - r.arrival for r in requests])
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "max_ms": float(lat.max() * 1e3)}

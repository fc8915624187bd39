"""Served form: request loops over the k-mer counter.

Count requests (a read set and k) arrive over time; each request's latency runs from its
arrival to the moment its result is complete on the device.  Two servers:

- serve_async (the served form): every arrived request whose device footprint fits what
  is left of the memory budget is submitted at once (kc_submit) and queued on the plan's
  stream, its scratch kept on the device; results are collected as they complete
  (kc_job_poll), so the GPU runs the requests back to back with no host round trip
  between them, and the host prepares and checks requests while the GPU counts.
- serve: rounds of kc_count_batch over the requests that arrived meanwhile (one call per
  k), for bursts of many requests.

No part of the counting happens here: this module only orders calls into the library.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

# device bytes per base a count needs at most: two key buffers of 8 or 16 bytes, the packed
# reads, the result buffers (keys + counts) and small per-tile / per-partition arrays
FOOTPRINT_PER_BASE = {1: 2 * 8 + 8 + 4 + 2, 2: 2 * 16 + 16 + 4 + 2}


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


def footprint(req: Request) -> int:
    return req.n_bases * FOOTPRINT_PER_BASE[1 if req.k <= 32 else 2] + (64 << 20)


def result_digest(res):
    """(distinct keys, valid windows, SHA-256 of the whole sorted result): two results have
    the same digest only if they hold the same keys with the same counts, entry by entry."""
    import hashlib
    keys, counts = res.to_numpy()
    h = hashlib.sha256()
    h.update(keys.tobytes())
    h.update(counts.tobytes())
    return (res.n, res.n_valid_windows, h.hexdigest())


def _finish(r: Request, res, t_done: float, keep_digest: bool):
    r.done = t_done
    r.n_distinct, r.n_valid = res.n, res.n_valid_windows
    if keep_digest:  # on the current stream: behind any counts still queued there
        r.digest = result_digest(res)
    res.free()


# service time a count is expected to take (ordering only): per base, by key width, plus a
# fixed part for the launches
SECONDS_PER_BASE = {1: 1.0 / 25e9, 2: 1.0 / 12e9}
SECONDS_FIXED = 0.3e-3


def expected_seconds(req: Request) -> float:
    return SECONDS_FIXED + req.n_bases * SECONDS_PER_BASE[1 if req.k <= 32 else 2]


def serve_async(counter, requests: list[Request], budget_bytes: int, canonical: bool = True,
                keep_digest: bool = True, idle_sleep: float = 50e-6, policy: str = "fifo", depth: int | None = None,
                batch: bool = False, max_batch: int = 64, batch_ratio: float = 4.0):
    """Submit arrived requests while the footprints of the requests in flight stay within the
    budget (and, with `depth`, while fewer than `depth` submissions are in flight); collect
    results as they complete.  One request is always admitted when none is in flight,
    whatever its footprint.  policy "fifo" takes the waiting requests in arrival order;
    "sjf" takes next the one with the least expected service time minus the time it has
    waited (shortest first, with ageing so that a large request is not held back for ever),
    and defaults to depth 2, so that the GPU always has the next submission queued.  With
    `batch` (continuous batching), the waiting requests with the same k whose expected
    service time is at most `batch_ratio` times that of the request taken (or under 1 ms)
    join it, in policy order and within the budget, in one submission of batched launches
    (kc_submit_batch, at most `max_batch` requests)."""
    if policy not in ("fifo", "sjf"):
        raise ValueError(f"unknown policy {policy!r}")
    if depth is None and policy == "sjf":
        depth = 2
    queue = collections.deque(sorted(requests, key=lambda r: r.arrival))
    waiting: list = []
    inflight: dict = {}  # job id -> (request, footprint, submission)
    open_subs: dict = {}  # submission -> its jobs still in flight
    next_sub = 0
    used = 0
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
            f = footprint(r)
            if inflight and used + f > budget_bytes:
                break
            group, tot = [i], used + f
            if batch:
                cap = max(batch_ratio * expected_seconds(r), 1e-3)
                for q in sorted((q for q in range(len(waiting)) if q != i and waiting[q].k == r.k), key=prio):
                    if len(group) >= max_batch:
                        break
                    fq = footprint(waiting[q])
                    if expected_seconds(waiting[q]) <= cap and tot + fq <= budget_bytes:
                        group.append(q)
                        tot += fq
            reqs = [waiting[q] for q in group]
            if len(reqs) == 1:
                jobs = [counter.submit(r.reads, r.offsets, r.k, canonical, n_bases=r.n_bases)]
            else:
                jobs = counter.submit_batch([(x.reads, x.offsets, x.n_bases) for x in reqs], r.k, canonical)
            open_subs[next_sub] = len(jobs)
            for job, x in zip(jobs, reqs):
                inflight[job] = (x, footprint(x), next_sub)
            next_sub += 1
            submissions += 1
            used = tot
            for q in sorted(group, reverse=True):
                waiting.pop(q)
        peak_inflight = max(peak_inflight, len(inflight))
        progressed = False
        for job in list(inflight):
            res = counter.poll(job)
            if res is None:
                continue
            r, f, sub = inflight.pop(job)
            used -= f
            open_subs[sub] -= 1
            if not open_subs[sub]:
                del open_subs[sub]
            _finish(r, res, time.perf_counter() - t0, keep_digest)
            progressed = True
        if not progressed:
            if not inflight and not waiting and queue:
                time.sleep(max(0.0, min(queue[0].arrival - (time.perf_counter() - t0), 0.002)))
            else:
                time.sleep(idle_sleep)
    return {"batches": submissions, "peak_inflight": peak_inflight, "makespan": time.perf_counter() - t0}


def serve(counter, requests: list[Request], budget_bytes: int, canonical: bool = True, keep_digest: bool = True):
    """Continuous batching in arrival order; fills done / n_distinct / n_valid / digest."""
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
        # admit in arrival order while the budget holds (at least one request per round)
        admitted, used = [], 0
        for r in waiting:
            f = footprint(r)
            if admitted and used + f > budget_bytes:
                continue
            admitted.append(r)
            used += f
        admitted_ids = {id(r) for r in admitted}
        waiting = [r for r in waiting if id(r) not in admitted_ids]
        by_k = collections.defaultdict(list)
        for r in admitted:
            by_k[r.k].append(r)
        for k, group in sorted(by_k.items()):
            results = counter.count_batch([(r.reads, r.offsets, r.n_bases) for r in group], k, canonical)
            t_done = time.perf_counter() - t0
            for r, res in zip(group, results):
                _finish(r, res, t_done, keep_digest)
            batches += 1
    return {"batches": batches, "makespan": time.perf_counter() - t0}


def serve_one_at_a_time(counter, requests: list[Request], canonical: bool = True, keep_digest: bool = True):
    """The plain loop: one kc_count per request, first come first served."""
    queue = sorted(requests, key=lambda r: r.arrival)
    t0 = time.perf_counter()
    for r in queue:
        now = time.perf_counter() - t0
        if r.arrival > now:
            time.sleep(r.arrival - now)
        res = counter.count(r.reads, r.offsets, r.k, canonical)
        _finish(r, res, time.perf_counter() - t0, keep_digest)
    return {"batches": len(queue), "makespan": time.perf_counter() - t0}


def latency_summary(requests: list[Request]) -> dict:
    lat = np.array([r.done - r.arrival for r in requests])
    return {"p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "mean_ms": float(lat.mean() * 1e3), "max_ms": float(lat.max() * 1e3)}

"""Autotuner for the plan options of the k-mer counter.

For a representative input, kc_count is timed (CUDA events on the plan's stream) under a
few plan options: the coarse partition count the library picks by itself, half and twice
that count, then the table load at the best count.  Every candidate must return the same
result (every key and count, compared on the device), and the fastest options are returned
for use with KmerCounter(**options) or count_batch on inputs of the same kind.
No part of the counting happens here: this module only times calls into the library.
"""
from __future__ import annotations

MAX_PARTITIONS = 4096
TABLE_LOADS = (0.45, 0.55)


class _DeviceResult:
    """A result's keys and counts, copied on the device; equal only if every key and count
    is (compared on the device, so that large results need no trip to the host)."""

    def __init__(self, res):
        self.keys = res.keys_tensor().clone()
        self.counts = res.counts_tensor().clone()
        self.n_valid = res.n_valid_windows

    def __eq__(self, other):
        import torch
        return (isinstance(other, _DeviceResult) and self.n_valid == other.n_valid
                and self.keys.shape == other.keys.shape and bool(torch.equal(self.keys, other.keys))
                and bool(torch.equal(self.counts, other.counts)))

    def __ne__(self, other):
        return not self.__eq__(other)


def _time_count(make_counter, opts, reads, offsets, k, canonical, repeats):
    """(median ms, the result, coarse partitions used) of kc_count under plan options `opts`."""
    import torch
    stream = torch.cuda.Stream()
    counter = make_counter(stream=stream, **opts)
    try:
        res = counter.count(reads, offsets, k, canonical)  # warm-up; its result is the check
        with torch.cuda.stream(stream):
            digest = _DeviceResult(res)
        stream.synchronize()
        res.free()
        p1 = counter.stats()["n_partitions"]
        times = []
        for _ in range(repeats):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            counter.count(reads, offsets, k, canonical).free()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        times.sort()
        return times[len(times) // 2], digest, p1
    finally:
        counter.close()


def autotune(reads, offsets, k: int, canonical: bool = True, repeats: int = 3, make_counter=None,
             timer=None) -> dict:
    """Fastest plan options for inputs like (reads, offsets) (device buffers for a fair timing).

    Returns {"best": options, "best_ms": ms, "trials": [(options, ms), ...]}.  `make_counter`
    builds a counter from plan options (default KmerCounter); `timer(options)` may replace the
    timing (it returns (ms, digest, partitions used))."""
    if make_counter is None:
        from . import KmerCounter
        make_counter = KmerCounter
    if timer is None:
        def timer(opts):
            return _time_count(make_counter, opts, reads, offsets, k, canonical, repeats)
    trials = []
    ref = None

    def run(opts):
        nonlocal ref
        ms, digest, p1 = timer(opts)
        if ref is None:
            ref = digest
        elif digest != ref:
            raise RuntimeError(f"plan options {opts} changed the result")
        trials.append((dict(opts), ms))
        return ms, p1

    # coarse partitions: the library's own choice, then half and twice that
    ms0, p1 = run({})
    best, best_ms = {}, ms0
    for p in (p1 // 2, p1 * 2):
        if 1 <= p <= MAX_PARTITIONS:
            ms, _ = run({"n_partitions_hint": p})
            if ms < best_ms:
                best, best_ms = {"n_partitions_hint": p}, ms
    # table load at the best partition count (0.55 is the library's default)
    for load in TABLE_LOADS:
        if load == 0.55:
            continue
        opts = dict(best, table_load=load)
        ms, _ = run(opts)
        if ms < best_ms:
            best, best_ms = opts, ms
    return {"best": best, "best_ms": best_ms, "trials": trials}

"""Benchmark: Gk-mers/s of the k-mer counter on a seeded synthetic workload.

One step = one kc_count (every kernel of the hot path) over the whole read set,
inputs resident in HBM.  Prints ONE JSON line (rank 0).  The timed steps run on a
plain plan; the per-kernel split behind the roofline figures comes from a separate
pass on a plan that records an event after every launch.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]
Under torchrun (N > 1) every rank counts its own replica of the workload on its
own GPU (no collective in the data path); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Gk-mers/s counted (bit-exact vs oracle), % HBM roofline; batched/served vs plain"
UNIT = "Gk-mers/s"
DEFAULT_WORKLOAD = "repeats_100mbp_150bp_30x_k31"
WORKLOAD_DESC = {
    "uniform_1mbp_100bp_10x_k31": "1 Mbp i.i.d. genome, 100 bp reads, 10x, 0.5% subst, 0.01% N, k=31 canonical",
    "repeats_100mbp_150bp_30x_k31": "100 Mbp genome (20% from 500 repeat families, Zipf 1.2, 2% divergence), "
                                    "150 bp reads, 30x, 0.5% subst, k=31 canonical",
    "long_50mbp_10kbp_20x_k63": "50 Mbp i.i.d. genome, log-normal 10 kbp reads, 20x, 5% errors 60/20/20, k=63 canonical",
    "batch_256_samples_k31": "256 samples: i.i.d. genomes log-uniform 0.1-50 Mbp (times --scale), 150 bp reads, "
                             "U(5,40)x, 0.5% subst, k=31 canonical (about 46 G bases); kc_count_batch in chunks "
                             "against the per-sample kc_count loop, plan options per sample-size class from the "
                             "autotuner",
}
BATCH_SEED = 1004  # seeds of the batched workload's samples: mix_seed(1004, i)
WORKLOAD_DESC["serve_2000_requests"] = (
    "2000 count requests, Poisson arrivals at 200/s, k uniform in {21, 31, 63}, read sets of genomes log-uniform "
    "0.05-20 Mbp (times --scale), 150 bp reads, U(10,30)x, 0.5% subst (drawn from a pool of 32 generated read sets); "
    "served by one plan: requests admitted while free device memory covers their footprint (kc_footprint), taken "
    "shortest expected first with ageing (kc_submit, queued on the plan's stream, two submissions in flight), "
    "completions polled (kc_job_poll), results handed to the client on the device; with continuous batching "
    "(waiting requests of the same k and similar size submitted together as batched launches, kc_submit_batch); "
    "against arrival order, rounds of kc_count_batch and one kc_count per request; latency at 200/s, throughput "
    "with all requests at once")
SERVE_SEED = 1005  # seeds of the served workload: pool read sets mix_seed(1005, i), arrivals RandomState(1005)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def source_hash():
    """Hash of the kernel source's code (comments and blank lines left out), so that a
    comment edit keeps the DRAM figures captured on that code."""
    import re
    h = hashlib.sha256()
    for f in ("kc_kernels.cu", "kc_internal.h"):
        with open(os.path.join(ROOT, "paper_2505_04431_gb300", "csrc", f), encoding="utf-8") as fh:
            text = re.sub(r"/\*.*?\*/", "", fh.read(), flags=re.S)
        for line in text.splitlines():
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def ncu_traffic(kernel, workload):
    """dram bytes per launch from the committed ncu summary, if taken on this kernel source."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            d = json.load(f)
        e = d.get(workload, {}).get(kernel)
        if e and e.get("source_hash") == source_hash():
            return float(e["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def max_over_ranks(x: float, dist=None, device=None) -> float:
    """The largest x over the ranks of the process group (x itself without one)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, world: int, steps: int, elapsed_ms: float) -> float:
    """Whole-job throughput in G units/s: every rank's units over the slowest rank's time."""
    return units_per_rank * world * steps / (elapsed_ms / 1e3) / 1e9


class Clocks:
    """nvidia-smi samples while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if not self.p:
            return None
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sms, mx, reasons = [], None, set()
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sms.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"), f[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sms)}


def kernel_bytes(L, n_reads, K, D, w):
    """algorithmic bytes per launch of each kernel: what the kernel must read and write at
    least (input bytes, offsets, packed codes, keys written to / read from their partition,
    the sorted output)"""
    packed = L // 4 + L // 8
    return {
        "k_pack_count": L + 8 * n_reads + packed,
        "k_scatter": packed + 8 * n_reads + K * w,
        "k_fine_hist": K * w,
        "k_fine_scatter": 2 * K * w,
        "k_count_emit": K * w + D * (w + 4),
    }


def _time_on_prefix(fn, reads, offsets, target_s):
    """(windows per s, sample text, seconds) of fn(reads, offsets) on the first reads of the
    workload, the prefix grown until one run takes at least target_s."""
    n = len(offsets) - 1
    m = max(1, n // 2000)
    while True:
        o = offsets[:m + 1]
        r = reads[: int(o[-1])]
        t0 = time.perf_counter()
        nv = fn(r, o)
        dt = time.perf_counter() - t0
        if dt >= target_s or m >= n:
            return nv / dt / 1e9, f"first {m} of {n} reads ({int(o[-1])} bases, {nv} windows), {dt:.1f} s", dt
        m = min(n, int(m * max(2.0, 1.2 * target_s / max(dt, 1e-3))))


def cpu_baseline(reads, offsets, k, target_s=8.0):
    """The oracle on the host cores: its multi-threaded variant on every core (the reported
    figure: read ranges counted in threads, merged by key with addition) and, beside it, the
    single-threaded definition, each on the first reads of the workload (about target_s of
    CPU work each)."""
    import oracle
    cores = os.cpu_count() or 1
    v1, s1, _ = _time_on_prefix(lambda r, o: oracle.count(r, o, k, True)[2], reads, offsets, target_s)
    vm, sm, _ = _time_on_prefix(lambda r, o: oracle.count_parallel(r, o, k, True, cores)[2], reads, offsets, target_s)
    return {"value": vm, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sm,
            "variant": "oracle.count_parallel: read ranges counted by the oracle in threads, merged by key",
            "single_thread": {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": s1}}


def run_reference(args):
    """--impl reference: the oracle (its multi-threaded variant on every host core) timed on
    a bounded sample of the workload per step."""
    import oracle
    import synth
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    reads, offsets, k = synth.workload(args.workload)
    n = len(offsets) - 1
    cores = os.cpu_count() or 1

    def run(r, o):
        return oracle.count_parallel(r, o, k, True, cores)[2]

    # size one step to ~6 s of CPU work
    m = max(1, n // 4000)
    while True:
        o = offsets[:m + 1]
        t0 = time.perf_counter()
        run(reads[: int(o[-1])], o)
        dt = time.perf_counter() - t0
        if dt >= 1.5 or m >= n:
            break
        m = min(n, m * 2)
    m = min(n, max(1, int(m * 6.0 / max(dt, 1e-3))))
    o = offsets[:m + 1]
    r = reads[: int(o[-1])]
    for _ in range(args.warmup):
        run(r, o)
    t0 = time.perf_counter()
    nv = 0
    for _ in range(args.steps):
        nv = run(r, o)
    dt = time.perf_counter() - t0
    value = nv * args.steps / dt / 1e9
    sample = f"first {m} of {n} reads ({int(o[-1])} bases, {nv} windows) per step"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64" if k <= 32 else "u128",
            "data": "synthetic", "config": {"workload": args.workload, "desc": WORKLOAD_DESC.get(args.workload, "")},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measure(workload, args, dist=None, world=1, rank=0, dev=0, with_e2e=True, with_cpu=True):
    """Time one workload on this rank: the timed steps on a plain plan (CUDA events on its
    stream), the per-kernel split from a separate profiled pass, the end-to-end figure
    through the public API with host buffers, and (rank 0) the CPU baseline.  Returns the
    JSON line's fields on rank 0, None elsewhere."""
    import torch
    import synth
    from paper_2505_04431_gb300 import KmerCounter

    reads, offsets, k = synth.workload(workload, args.scale)
    n_reads, L = len(offsets) - 1, len(reads)
    stream = torch.cuda.Stream(dev)
    counter = KmerCounter(device=dev, stream=stream)  # the product path: no per-launch events
    r_dev = torch.from_numpy(reads).to(dev)
    o_dev = torch.from_numpy(offsets.view(np.int64)).to(dev)
    torch.cuda.synchronize()

    def step(c=counter):
        res = c.count(r_dev, o_dev, k, True)
        out = (res.n, res.n_valid_windows, res.key_words)
        res.free()
        return out

    for _ in range(args.warmup):
        step()
    clocks = Clocks(dev)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_wall = time.perf_counter()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    launches = 0
    D = K = kw = 0
    for _ in range(args.steps):
        D, K, kw = step()
        launches += counter.stats()["kernel_launches"]
    ev1.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    stats = counter.stats()
    elapsed_ms = max_over_ranks(ev0.elapsed_time(ev1), dist, dev)
    if dist:
        dist.barrier()
    ms_per_step = elapsed_ms / args.steps
    value = whole_job_rate(K, world, args.steps, elapsed_ms)

    # end to end through the public API with host buffers.  Pipelined (the value): kc_submit
    # of the pinned host reads (copied in on the plan's transfer stream) and
    # kc_job_copy_to_host of each result into pinned host buffers (copied out there as soon as
    # the count ends), two counts in flight, so that the copies of one step overlap the
    # counting of the next.  Serial (reported beside it): kc_count with the host buffers, then
    # kc_result_copy_to_host, one step at a time, with its parts timed apart.  Both run on the
    # plan of the timed steps, before the profiled pass: a plan in steady use, its scratch and
    # result blocks already held by the caching allocator.
    e2e = None
    if with_e2e and not args.no_e2e:
        import collections
        import ctypes
        from paper_2505_04431_gb300 import load_library, _check
        lib = load_library()
        r_pin = torch.from_numpy(reads).pin_memory()
        o_pin = torch.from_numpy(offsets.view(np.int64)).pin_memory()
        outs = [(torch.empty(max(1, D * kw), dtype=torch.int64).pin_memory(),
                 torch.empty(max(1, D), dtype=torch.int32).pin_memory()) for _ in range(2)]

        def link_probe():
            """The host link as it is now: the reads copied in from and out to their pinned
            buffer (the device copy holds the same bytes), best of two, on the plan's stream."""
            out = {}
            for name, dst, src in (("h2d", r_dev, r_pin), ("d2h", r_pin, r_dev)):
                best = float("inf")
                for _ in range(2):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    with torch.cuda.stream(stream):
                        e0.record(stream)
                        dst.copy_(src, non_blocking=True)
                        e1.record(stream)
                    stream.synchronize()
                    best = min(best, e0.elapsed_time(e1))
                out[name] = L / best / 1e6
            return out

        def pipelined(n):
            jobs = collections.deque()
            got = 0
            for i in range(n):
                if len(jobs) == 2:
                    res = counter.wait(jobs.popleft())
                    got += res.n
                    res.free()
                j = counter.submit(r_pin, o_pin, k, True, n_bases=L)
                counter.copy_to_host(j, *outs[i % 2])
                jobs.append(j)
            while jobs:
                res = counter.wait(jobs.popleft())
                got += res.n
                res.free()
            return got

        e2e_steps = max(3, args.steps)  # as many steps as the device-resident timing
        e2e_warmup = max(3, args.warmup)
        link_before = link_probe()
        pipelined(e2e_warmup)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        got = pipelined(e2e_steps)
        dt_pipe = max_over_ranks(time.perf_counter() - t0, dist, dev)
        if got != D * e2e_steps:
            raise RuntimeError(f"pipelined counts returned {got} entries, expected {D * e2e_steps}")
        keys_h, cnt_h = outs[0]

        # each serial step timed in its own parts as it runs: the count call (its input copy
        # included) and the result copy, device time by events on the plan's stream and host
        # wall clock around each call
        steps_parts = []

        def serial_step():
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            t_a = time.perf_counter()
            ev[0].record(stream)
            res = counter.count(r_pin, o_pin, k, True)
            ev[1].record(stream)
            t_b = time.perf_counter()
            _check(lib, lib.kc_result_copy_to_host(counter._plan, ctypes.byref(res._res), keys_h.data_ptr(),
                                                   cnt_h.data_ptr()))
            ev[2].record(stream)
            t_c = time.perf_counter()
            res.free()
            steps_parts.append((ev, (t_b - t_a) * 1e3, (t_c - t_b) * 1e3, (time.perf_counter() - t_c) * 1e3, t_a))

        for _ in range(e2e_warmup):
            serial_step()
        torch.cuda.synchronize()
        steps_parts.clear()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            serial_step()
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0, dist, dev)
        sp = np.array([(ev[0].elapsed_time(ev[1]), wa, ev[1].elapsed_time(ev[2]), wb, wf) for ev, wa, wb, wf, _ in steps_parts])
        starts = [x[4] for x in steps_parts]
        in_step = {"count_call_device_ms": float(np.median(sp[:, 0])), "count_call_wall_ms": float(np.median(sp[:, 1])),
                   "copy_out_device_ms": float(np.median(sp[:, 2])), "copy_out_wall_ms": float(np.median(sp[:, 3])),
                   "free_wall_ms": float(np.median(sp[:, 4])),
                   "step_wall_ms": float(np.median(np.diff(starts)) * 1e3) if len(starts) > 1 else None}
        # the serial step's parts apart, host wall clock around each with the stream drained:
        # the inputs in (the same pinned buffers), the count on those device inputs, the result out
        rd = torch.empty_like(r_pin, device=dev)
        od = torch.empty_like(o_pin, device=dev)
        reps = []
        for _ in range(4):
            torch.cuda.synchronize()
            t_a = time.perf_counter()
            with torch.cuda.stream(stream):
                rd.copy_(r_pin, non_blocking=True)
                od.copy_(o_pin, non_blocking=True)
            stream.synchronize()
            t_b = time.perf_counter()
            res = counter.count(rd, od, k, True)
            t_c = time.perf_counter()
            _check(lib, lib.kc_result_copy_to_host(counter._plan, ctypes.byref(res._res), keys_h.data_ptr(),
                                                   cnt_h.data_ptr()))
            t_d = time.perf_counter()
            res.free()
            reps.append(((t_b - t_a) * 1e3, (t_c - t_b) * 1e3, (t_d - t_c) * 1e3))
        med = np.median(np.array(reps[1:]), axis=0)
        parts = {"h2d_ms": float(med[0]), "count_ms": float(med[1]), "d2h_ms": float(med[2])}
        parts["rest_ms"] = dt * 1e3 / e2e_steps - sum(parts.values())
        del rd, od
        link_after = link_probe()
        h2d_bytes = int(L + 8 * (n_reads + 1))
        d2h_bytes = int(D * (8 * kw + 4))
        e2e = {"value": whole_job_rate(K, world, e2e_steps, dt_pipe * 1e3), "unit": UNIT,
               "h2d_bytes_per_step": h2d_bytes, "d2h_bytes_per_step": d2h_bytes,
               "steps": e2e_steps, "ms_per_step": dt_pipe * 1e3 / e2e_steps,
               "form": "kc_submit (pinned host reads, copied in on the transfer stream) + kc_job_copy_to_host "
                       "(result to pinned host buffers) + kc_job_wait, two counts in flight",
               "serial": {"value": whole_job_rate(K, world, e2e_steps, dt * 1e3), "ms_per_step": dt * 1e3 / e2e_steps,
                          "form": "kc_count (pinned host reads) + kc_result_copy_to_host, one step at a time",
                          "parts": parts, "in_step": in_step,
                          "link_gbs": {"h2d": h2d_bytes / parts["h2d_ms"] / 1e6,
                                       "d2h": d2h_bytes / max(parts["d2h_ms"], 1e-9) / 1e6}},
               "link_probe_gbs": {"before": link_before, "after": link_after,
                                  "what": f"the {L / 1e9:.2f} GB of reads copied in and out alone, best of two, "
                                          "before the pipelined run and after the serial one"}}
        del r_pin, o_pin, outs, keys_h, cnt_h

    counter.close()
    torch.cuda.empty_cache()
    # per-kernel split: the same steps on a plan that records a CUDA event on its stream after
    # every launch (a separate pass, so that the timed steps above run the plain product path)
    pstream = torch.cuda.Stream(dev)
    pcounter = KmerCounter(device=dev, stream=pstream, profile=True)
    step(pcounter)
    ktimes = {}
    prof_steps = max(3, min(args.steps, 5))
    for _ in range(prof_steps):
        step(pcounter)
        for name, ms in pcounter.kernel_times():
            ktimes.setdefault(name, []).append(ms)
    pcounter.close()
    torch.cuda.empty_cache()
    # pinned host buffers cached by torch go back to the system too, so that the next
    # workload's end-to-end run does not sit beside them
    torch.cuda.synchronize()
    if hasattr(torch._C, "_host_emptyCache"):
        torch._C._host_emptyCache()
    if rank != 0:
        return None
    w = 8 * kw
    peak, peak_kind = measured_peaks()
    kb = kernel_bytes(L, n_reads, K, D, w)
    avg = {n: sum(v) / len(v) for n, v in ktimes.items()}
    total_k = sum(avg.values()) or 1.0
    dom = max((n for n in avg if n in kb), key=lambda n: avg[n])
    achieved = kb[dom] / (avg[dom] / 1e3) / 1e9
    B = L + 8 * n_reads + 2 * K * w + D * (w + 4)
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": f"{peak_kind} hbm_gbs", "traffic": ncu_traffic(dom, workload),
                "alg_bytes_per_launch": kb[dom], "ms_per_launch": avg[dom], "share": avg[dom] / total_k,
                "timing": f"CUDA events on the plan's stream around every launch, {prof_steps} profiled steps"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64" if kw == 1 else "u128", "data": "synthetic",
        "config": {"workload": workload, "desc": WORKLOAD_DESC.get(workload, ""), "k": k, "canonical": True,
                   "reads": n_reads, "bases": L, "windows": K, "distinct": D,
                   "l2": f"inputs larger than L2 ({L / 1e9:.2f} GB of reads, {K * w / 1e9:.1f} GB of keys per step)",
                   "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
        "roofline": roofline,
        "path_roofline": {"bytes": B, "achieved": B / (ms_per_step / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                          "frac": B / (ms_per_step / 1e3) / 1e9 / peak},
        "kernels_ms": {n: round(v, 4) for n, v in sorted(avg.items(), key=lambda x: -x[1])},
        "gpu_launches": launches,
        "stats": stats,
        "clocks": clk,
        "e2e": e2e,
        "wall_s": wall,
    }
    if world == 1 and with_cpu == "defer" and not args.no_cpu_baseline:
        line["_cpu_inputs"] = (reads, offsets, k)  # timed after every GPU measurement
    elif world == 1 and with_cpu and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(reads, offsets, k)
    return line


def run_ours(args):
    import torch
    from paper_2505_04431_gb300 import build as kcbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    if rank == 0:
        kcbuild.build()
    if dist:
        dist.barrier()
    with_extras = world == 1 and not args.no_extras and args.workload == DEFAULT_WORKLOAD
    # with the extra forms, the oracle on the host cores runs last, after all GPU work, so that
    # its threads and host memory sit beside none of the end-to-end runs
    line = measure(args.workload, args, dist, world, rank, dev, with_cpu="defer" if with_extras else True)
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return
    # the other forms, as extra keys of the same line (one GPU; each after the device memory
    # of the one before is released)
    if with_extras:
        extras = {}
        for key, fn in (("long_50mbp_10kbp_20x_k63",
                         lambda: measure("long_50mbp_10kbp_20x_k63", args, dev=dev, with_cpu=False)),
                        ("batched", lambda: run_batch(args, as_summary=True)),
                        ("served", lambda: run_serve(args, as_summary=True))):
            torch.cuda.empty_cache()
            t0 = time.perf_counter()
            try:
                extras[key] = fn()
                extras[key]["seconds"] = time.perf_counter() - t0
            except Exception as exc:  # recorded, so that the headline line is still printed
                extras[key] = {"error": f"{type(exc).__name__}: {exc}"}
        k63 = extras.get("long_50mbp_10kbp_20x_k63", {})
        if "value" in k63:
            extras["long_50mbp_10kbp_20x_k63"] = {
                kk: k63[kk] for kk in ("value", "unit", "ms_per_step", "roofline", "path_roofline", "kernels_ms",
                                       "e2e", "config", "clocks", "seconds") if kk in k63}
        line["other_workloads"] = extras
    cpu_inputs = line.pop("_cpu_inputs", None)
    if cpu_inputs is not None:
        line["cpu_baseline"] = cpu_baseline(*cpu_inputs)
    print(json.dumps(line), flush=True)


def run_batch(args, as_summary=False):
    """The batched form against the plain per-sample loop on the 256 samples of the batched
    workload (genomes log-uniform 0.1-50 Mbp at 5-40x, about 46 G bases at --scale 1),
    streamed through the GPU in chunks of samples whose results fit device memory, both
    timed end to end on the host (wall clock around all calls, inputs resident on the
    device, results freed as each chunk is done).  Plan options per sample-size class come
    from the autotuner; untimed, every sample's result from the batch is compared on the
    device, key for key and count for count, with its count alone."""
    import concurrent.futures as cf
    import torch
    import synth
    from paper_2505_04431_gb300 import KmerCounter
    from paper_2505_04431_gb300 import build as kcbuild
    from paper_2505_04431_gb300 import tune

    torch.cuda.set_device(0)
    kcbuild.build()
    scale = args.scale
    samples = []
    with cf.ThreadPoolExecutor(min(32, os.cpu_count() or 4)) as ex:
        for r, o, _ in ex.map(lambda i: synth.generate(synth.SAMPLE, synth.mix_seed(BATCH_SEED, i), scale), range(256)):
            samples.append((torch.from_numpy(r).cuda(), torch.from_numpy(o.view(np.int64)).cuda(), int(o[-1])))
    torch.cuda.synchronize()
    bases = sum(s_[2] for s_ in samples)
    # size classes, each with the plan options the autotuner picks on its median sample
    cuts = (1 << 26, 1 << 29)  # 64 Mi, 512 Mi bases
    cls = [sum(s_[2] >= c for c in cuts) for s_ in samples]
    tuned, counters = {}, {}
    for c in sorted(set(cls)):
        members = sorted((i for i in range(len(samples)) if cls[i] == c), key=lambda i: samples[i][2])
        med = samples[members[len(members) // 2]]
        t = tune.autotune(med[0], med[1], 31, True, repeats=2)
        tuned[c] = {"options": t["best"], "best_ms": t["best_ms"], "samples": len(members),
                    "tuned_on_bases": med[2]}
        counters[c] = KmerCounter(**t["best"])
    # chunks of consecutive samples of one class whose result buffers stay within a budget
    budget = 48 << 30
    order = sorted(range(len(samples)), key=lambda i: (cls[i], samples[i][2]))
    chunks, cur, used = [], [], 0
    for i in order:
        need = samples[i][2] * 12
        if cur and (used + need > budget or cls[cur[0]] != cls[i]):
            chunks.append(cur)
            cur, used = [], 0
        cur.append(i)
        used += need
    if cur:
        chunks.append(cur)

    def batched(check=False):
        v, bad = 0, []
        for ch in chunks:
            c = counters[cls[ch[0]]]
            out = c.count_batch([samples[i] for i in ch], 31, True)
            v += sum(res.n_valid_windows for res in out)
            for i, res in zip(ch, out):
                if check:
                    alone = c.count(samples[i][0], samples[i][1], 31, True)
                    if not _same(res, (alone.keys_tensor(), alone.counts_tensor(), alone.n_valid_windows)):
                        bad.append(i)
                    alone.free()
                res.free()
        return v, bad

    def plain():
        v = 0
        for ch in chunks:
            c = counters[cls[ch[0]]]
            for i in ch:
                res = c.count(samples[i][0], samples[i][1], 31, True)
                v += res.n_valid_windows
                res.free()
        return v

    # checked once (not timed): every sample's result from the batch equals its count alone
    _, bad = batched(check=True)
    if bad:
        raise RuntimeError(f"batched results differ from kc_count alone for {len(bad)} samples (first: {bad[0]})")
    t_plain, t_batch, valid = [], [], 0
    for it in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        v1 = plain()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        v2, _ = batched()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        if v1 != v2:
            raise RuntimeError(f"batched and plain counts differ in valid windows: {v1} vs {v2}")
        valid = v1
        if it >= args.warmup:
            t_plain.append(t1 - t0)
            t_batch.append(t2 - t1)
    tp, tb = float(np.median(t_plain)), float(np.median(t_batch))
    launches = sum(c.stats()["kernel_launches"] for c in counters.values())
    # small samples alone: 256 samples of about 0.4 M bases, where launches dominate
    small = []
    for i in range(256):
        r, o, _ = synth.generate(synth.SAMPLE, synth.mix_seed(BATCH_SEED + 1, i), 0.002)
        small.append((torch.from_numpy(r).cuda(), torch.from_numpy(o.view(np.int64)).cuda(), int(o[-1])))
    c0 = KmerCounter()
    sw = sum(s_[2] for s_ in small)

    def small_runs():
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        v = 0
        for s_ in small:
            res = c0.count(s_[0], s_[1], 31, True)
            v += res.n_valid_windows
            res.free()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        out = c0.count_batch(small, 31, True)
        w = sum(res.n_valid_windows for res in out)
        for res in out:
            res.free()
        torch.cuda.synchronize()
        return t1 - t0, time.perf_counter() - t1, v, w

    small_runs()
    sp, sb, sv_, sw_ = small_runs()
    c0.close()
    for c in counters.values():
        c.close()
    out = {"samples": len(samples), "genome_scale": scale, "bases": bases, "windows": valid, "chunks": len(chunks),
           "batched": {"value": valid / tb / 1e9, "unit": UNIT, "ms_per_step": tb * 1e3},
           "plain": {"value": valid / tp / 1e9, "unit": UNIT, "ms_per_step": tp * 1e3},
           "batched_vs_plain": tp / tb, "size_classes": {str(k): v for k, v in tuned.items()},
           "small_samples": {"samples": len(small), "bases": sw, "plain_ms": sp * 1e3, "batched_ms": sb * 1e3,
                             "batched_vs_plain": sp / sb, "plain_launches": 13 * len(small)},
           "results_identical": True, "gpu_launches": launches}
    if as_summary:
        return out
    line = {"metric": METRIC, "value": valid / tb / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tb * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": WORKLOAD_DESC[args.workload], "k": 31, "canonical": True,
                       "parallelism": "1 GPU", "timing": "host wall clock around all calls, median of steps"},
            "batch": out, "gpu_launches": launches}
    print(json.dumps(line), flush=True)


def _device_copy(res):
    """The used part of a result, copied into tensors of its own (kept while results come and go)."""
    return res.keys_tensor().clone(), res.counts_tensor().clone(), res.n_valid_windows


def _same(res, ref) -> bool:
    """Every key and count of a result equals the reference's (compared on the device)."""
    import torch
    return (res.n_valid_windows == ref[2] and res.n == ref[1].shape[0]
            and bool(torch.equal(res.keys_tensor(), ref[0])) and bool(torch.equal(res.counts_tensor(), ref[1])))


def run_serve(args, as_summary=False):
    """The served form against the plain loop on one arrival sequence of 2000 requests:
    latency at 200 requests/s (Poisson), throughput with all requests arriving at once
    (saturation), and, untimed, every request's result compared key for key and count for
    count with the same count alone."""
    import torch
    import synth
    from paper_2505_04431_gb300 import KmerCounter
    from paper_2505_04431_gb300 import build as kcbuild
    from paper_2505_04431_gb300 import serve as sv

    torch.cuda.set_device(0)
    kcbuild.build()
    import concurrent.futures as cf
    with cf.ThreadPoolExecutor(min(32, os.cpu_count() or 4)) as ex:
        gen = list(ex.map(lambda i: synth.generate(synth.SERVE, synth.mix_seed(SERVE_SEED, i), args.scale), range(32)))
    pool = [(torch.from_numpy(r).cuda(), torch.from_numpy(o.view(np.int64)).cuda(), int(o[-1])) for r, o, _ in gen]
    del gen
    torch.cuda.synchronize()
    rng = np.random.RandomState(SERVE_SEED)
    n_req, rate = 2000, 200.0
    arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
    ks = rng.choice([21, 31, 63], n_req)
    picks = rng.randint(0, len(pool), n_req)

    def make(at_once=False):
        return [sv.Request(0.0 if at_once else float(a), pool[p][0], pool[p][1], pool[p][2], int(k))
                for a, k, p in zip(arrivals, ks, picks)]

    counter = KmerCounter()
    # the result of every (read set, k) of the mix, counted alone and kept on the device
    ref = {}
    for p_, k_ in sorted(set(zip(picks.tolist(), ks.tolist()))):
        res = counter.count(pool[p_][0], pool[p_][1], k_)
        ref[(p_, k_)] = _device_copy(res)
        res.free()
    torch.cuda.synchronize()
    free_result = lambda r, res: res.free()  # noqa: E731  (the client is done with it)
    servers = {
        "served": lambda reqs: sv.serve_async(counter, reqs, keep_digest=False, policy="sjf", on_result=free_result),
        "served_batched": lambda reqs: sv.serve_async(counter, reqs, keep_digest=False, policy="sjf", batch=True,
                                                      on_result=free_result),
        "served_fifo": lambda reqs: sv.serve_async(counter, reqs, keep_digest=False, policy="fifo",
                                                   on_result=free_result),
        "batch_rounds": lambda reqs: sv.serve(counter, reqs, keep_digest=False, on_result=free_result),
        "plain": lambda reqs: sv.serve_one_at_a_time(counter, reqs, keep_digest=False, on_result=free_result),
    }
    servers["served_batched"](make(True))  # warm-up: every k and size once, scratch grown
    runs, sat = {}, {}
    for name, fn in servers.items():
        reqs = make()
        torch.cuda.synchronize()
        runs[name] = (reqs, fn(reqs))
    for name in ("served_batched", "served", "plain"):
        reqs = make(True)
        torch.cuda.synchronize()
        sat[name] = (reqs, servers[name](reqs))
    # checked (not timed): every request's result in the mix equals the same count alone
    checked = 0
    for name in ("served", "served_batched", "batch_rounds"):
        bad = []

        def check(r, res, bad=bad):
            if not _same(res, ref[(r._pick, r.k)]):
                bad.append(r)
            res.free()

        reqs = make(True)
        for r, p_ in zip(reqs, picks):
            r._pick = int(p_)
        if name == "batch_rounds":
            sv.serve(counter, reqs, keep_digest=False, on_result=check)
        else:
            sv.serve_async(counter, reqs, keep_digest=False, policy="sjf", batch=name == "served_batched",
                           on_result=check)
        if bad:
            raise RuntimeError(f"{name}: {len(bad)} results differ from the same count alone")
        checked += len(reqs)
    windows = sum(r.n_valid for r in runs["served"][0])

    def summary(reqs, info):
        return {"value": windows / info["makespan"] / 1e9, "unit": UNIT, "ms_per_step": info["makespan"] * 1e3,
                "latency": sv.latency_summary(reqs), "submissions": info["batches"]}

    lat = {n: summary(*runs[n]) for n in runs}
    thr = {n: summary(*sat[n]) for n in sat}
    out = {"requests": n_req, "rate_per_s": rate, "windows": windows,
           "offered_gkmers_per_s": windows / float(arrivals[-1]) / 1e9,
           "at_200_per_s": {n: {"p50_ms": v["latency"]["p50_ms"], "p99_ms": v["latency"]["p99_ms"],
                                "gkmers_per_s": v["value"], "submissions": v["submissions"]} for n, v in lat.items()},
           "saturated": {n: {"gkmers_per_s": v["value"], "makespan_ms": v["ms_per_step"],
                             "submissions": v["submissions"]} for n, v in thr.items()},
           "served_over_plain_saturated": thr["served_batched"]["value"] / thr["plain"]["value"],
           "results_checked": checked, "results_identical": True}
    counter.close()
    if as_summary:
        return out
    line = {"metric": METRIC, "value": thr["served_batched"]["value"], "unit": UNIT, "n_gpus": 1, "steps": 1,
            "warmup": 1, "ms_per_step": thr["served_batched"]["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64/u128", "data": "synthetic",
            "config": {"workload": args.workload, "desc": WORKLOAD_DESC[args.workload], "genome_scale": args.scale,
                       "parallelism": "1 GPU",
                       "timing": "host wall clock; latency = arrival to the host seeing the count complete; value = "
                                 "windows / makespan with all 2000 requests arriving at once"},
            "served": out, "gpu_launches": 13 * n_req}
    print(json.dumps(line), flush=True)


WORKLOAD_DESC["ablation_aggregation"] = (
    "aggregation ablation (the GPU analogue of adding the paper's L2 and L3 layers one at a time) on "
    "uniform_1mbp_100bp_10x_k31 and repeats_100mbp_150bp_30x_k31: L0-L1 = pass B writes every key on its own "
    "through global atomic cursors and the count kernel adds every key on its own; L0-L2 = shared-memory "
    "buckets in pass B (the default); L0-L3 = and the warp merge of equal keys in the count kernel")
ABLATION_VARIANTS = (("L0-L1", True, False), ("L0-L3", False, True), ("L0-L2", False, False))  # the default last


def run_ablation(args):
    """Each aggregation variant timed like the plain counter (CUDA events on the plan's stream,
    inputs in HBM), on configs 1 and 2; every variant's result digest must equal the default's."""
    import torch
    import synth
    from paper_2505_04431_gb300 import KmerCounter
    from paper_2505_04431_gb300 import build as kcbuild
    from paper_2505_04431_gb300 import serve as sv

    torch.cuda.set_device(0)
    kcbuild.build()
    out = {}
    launches = 0
    for wl in ("uniform_1mbp_100bp_10x_k31", "repeats_100mbp_150bp_30x_k31"):
        reads, offsets, k = synth.workload(wl, args.scale)
        r_dev = torch.from_numpy(reads).cuda()
        o_dev = torch.from_numpy(offsets.view(np.int64)).cuda()
        torch.cuda.synchronize()
        res_wl, ref = {}, None
        for name, no_buckets, merge in reversed(ABLATION_VARIANTS):  # the default first: the reference
            stream = torch.cuda.Stream()
            c = KmerCounter(stream=stream, profile=True, no_smem_buckets=no_buckets, warp_merge=merge)
            res = c.count(r_dev, o_dev, k, True)
            dig = sv.result_digest(res)
            res.free()
            if ref is None:
                ref = dig
            elif dig != ref:
                raise RuntimeError(f"{wl} {name}: result differs from the default")
            for _ in range(args.warmup):
                c.count(r_dev, o_dev, k, True).free()
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ktimes = {}
            ev0.record(stream)
            for _ in range(args.steps):
                c.count(r_dev, o_dev, k, True).free()
                launches += c.stats()["kernel_launches"]
                for kn, ms in c.kernel_times():
                    ktimes.setdefault(kn, []).append(ms)
            ev1.record(stream)
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1) / args.steps
            kms = {kn: sum(v) / len(v) for kn, v in ktimes.items()}
            res_wl[name] = {"value": dig[1] / (ms / 1e3) / 1e9, "ms_per_step": ms,
                            "pass_b_ms": kms.get("k_scatter", 0.0) + kms.get("k_direct_cursors", 0.0),
                            "count_ms": kms.get("k_count_emit", 0.0)}
            c.close()
        base = res_wl["L0-L1"]["ms_per_step"]
        for name in res_wl:
            res_wl[name]["speedup_over_L0_L1"] = base / res_wl[name]["ms_per_step"]
        out[wl] = res_wl
    head = out["repeats_100mbp_150bp_30x_k31"]["L0-L2"]
    line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": WORKLOAD_DESC[args.workload], "genome_scale": args.scale,
                       "parallelism": "1 GPU", "timing": "CUDA events on the plan's stream, per-kernel events"},
            "ablation": out, "results_identical": True, "gpu_launches": launches}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOAD_DESC))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="the headline workload only (no k=63, batched and served summaries)")
    ap.add_argument("--scale", type=float, default=1.0, help="genome scale (diagnostics only; 1.0 = the workload)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        run_reference(args)
    elif args.workload.startswith("batch_"):
        run_batch(args)
    elif args.workload.startswith("serve_"):
        run_serve(args)
    elif args.workload == "ablation_aggregation":
        run_ablation(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

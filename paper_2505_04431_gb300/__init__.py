"""GB300-native k-mer counter: Python binding of the C ABI in include/kc.h.

This module only marshals arguments: every step of the count runs in the CUDA
kernels of libkc.so (built in-tree by build.py).  PyTorch provides device
memory (its caching allocator, through the plan's alloc/free hooks) and the
current CUDA stream.  There is no CPU fallback: without the built library, or
without a CUDA device, the calls raise.

    counter = KmerCounter()                       # plan on the current device/stream
    res = counter.count(reads, offsets, k=31)     # reads: uint8, offsets: uint64 (n_reads + 1)
    keys, counts = res.to_numpy()                 # ascending keys, their counts
    res.free()
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkc.so")

KC_OK, KC_EINVAL, KC_ENOMEM, KC_ECUDA, KC_EOVERFLOW, KC_ETIMEOUT, KC_EBUSY = range(7)
STATUS_NAMES = {0: "KC_OK", 1: "KC_EINVAL", 2: "KC_ENOMEM", 3: "KC_ECUDA", 4: "KC_EOVERFLOW",
                5: "KC_ETIMEOUT", 6: "KC_EBUSY"}

# every entry point declared in include/kc.h
EXPORTED = ["kc_plan", "kc_count", "kc_free", "kc_result_copy_to_host", "kc_plan_destroy",
            "kc_last_error", "kc_last_stats", "kc_last_kernel_times", "kc_count_noalloc", "kc_count_batch",
            "kc_submit", "kc_job_poll", "kc_job_wait", "kc_submit_batch", "kc_footprint",
            "kc_job_copy_to_host"]
KC_NOALLOC_MAX_BASES = 1 << 20
KC_PLAN_PROFILE = 1
KC_PLAN_DEFER_ALL = 2
KC_PLAN_BATCH_ARENA_SMALL = 4
KC_PLAN_ABLATE_NO_SMEM_BUCKETS = 8
KC_PLAN_WARP_MERGE = 16
KC_PLAN_TEST_WITHHOLD_PREFIX = 32
KC_PLAN_TEST_COUNT_LIMIT = 64
KC_PLAN_TEST_FINE_SAMPLED = 128
KC_PLAN_TEST_TIGHT_SLACK = 256

_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class PlanOpts(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("stream", ctypes.c_void_p),
                ("alloc", _ALLOC_FN), ("free_", _FREE_FN), ("alloc_ctx", ctypes.c_void_p),
                ("max_device_bytes", ctypes.c_uint64), ("n_partitions_hint", ctypes.c_uint32),
                ("block_size_hint", ctypes.c_uint32), ("table_load", ctypes.c_float),
                ("table_slots_max", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


class Result(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("key_words", ctypes.c_uint32), ("keys", ctypes.c_void_p),
                ("counts", ctypes.c_void_p), ("n_valid_windows", ctypes.c_uint64),
                ("capacity", ctypes.c_uint64), ("_owner", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_uint32), ("n_partitions", ctypes.c_uint32),
                ("n_fine", ctypes.c_uint64), ("n_overflow_fine", ctypes.c_uint64), ("n_deferred_fine", ctypes.c_uint64),
                ("workspace_bytes", ctypes.c_uint64), ("phase_cycles", ctypes.c_uint64 * 8),
                ("sub_cycles", ctypes.c_uint64 * 8), ("fine_sampled", ctypes.c_uint32),
                ("fine_resplit", ctypes.c_uint32)]


class KcError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libkc.so and declare its signatures.  Raises if it was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libkc.so not found at {path}; build it with paper_2505_04431_gb300.build.build()")
    lib = ctypes.CDLL(path)
    vp, u64, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
    lib.kc_plan.argtypes = [ctypes.POINTER(PlanOpts), ctypes.POINTER(vp)]
    lib.kc_plan.restype = i32
    lib.kc_count.argtypes = [vp, vp, vp, u64, i32, i32, ctypes.POINTER(Result)]
    lib.kc_count.restype = i32
    lib.kc_free.argtypes = [vp, ctypes.POINTER(Result)]
    lib.kc_free.restype = i32
    lib.kc_result_copy_to_host.argtypes = [vp, ctypes.POINTER(Result), vp, vp]
    lib.kc_result_copy_to_host.restype = i32
    lib.kc_plan_destroy.argtypes = [vp]
    lib.kc_plan_destroy.restype = i32
    lib.kc_last_error.argtypes = []
    lib.kc_last_error.restype = ctypes.c_char_p
    lib.kc_last_stats.argtypes = [vp, ctypes.POINTER(Stats)]
    lib.kc_last_stats.restype = i32
    lib.kc_last_kernel_times.argtypes = [vp, ctypes.c_uint32, ctypes.POINTER(ctypes.c_char_p),
                                         ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_uint32)]
    lib.kc_last_kernel_times.restype = i32
    lib.kc_count_noalloc.argtypes = [vp, vp, u64, i32, i32, vp, vp, u64, ctypes.POINTER(u64), ctypes.POINTER(u64), vp]
    lib.kc_count_noalloc.restype = i32
    P = ctypes.POINTER
    lib.kc_count_batch.argtypes = [vp, ctypes.c_uint32, P(vp), P(vp), P(u64), P(u64), i32, i32, P(Result)]
    lib.kc_count_batch.restype = i32
    lib.kc_submit.argtypes = [vp, vp, vp, u64, u64, i32, i32, P(u64)]
    lib.kc_submit.restype = i32
    lib.kc_job_poll.argtypes = [vp, u64, P(Result), P(i32)]
    lib.kc_job_poll.restype = i32
    lib.kc_job_wait.argtypes = [vp, u64, P(Result)]
    lib.kc_job_wait.restype = i32
    lib.kc_submit_batch.argtypes = [vp, ctypes.c_uint32, P(vp), P(vp), P(u64), P(u64), i32, i32, P(u64)]
    lib.kc_submit_batch.restype = i32
    lib.kc_footprint.argtypes = [vp, u64, u64, i32, i32, i32, P(u64), P(u64)]
    lib.kc_footprint.restype = i32
    lib.kc_job_copy_to_host.argtypes = [vp, u64, vp, vp, u64]
    lib.kc_job_copy_to_host.restype = i32
    _lib = lib
    return lib


def _check(lib, st: int):
    if st != KC_OK:
        raise KcError(st, (lib.kc_last_error() or b"").decode())


def _ptr(x):
    """(pointer, keepalive) for a numpy array or torch tensor (host or device)."""
    if isinstance(x, np.ndarray):
        x = np.ascontiguousarray(x)
        return x.ctypes.data, x
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            x = x.contiguous()
        return x.data_ptr(), x
    raise TypeError(f"unsupported buffer type {type(x)}")


class _DeviceArray:
    """Exposes a device buffer through __cuda_array_interface__ (no copy)."""

    def __init__(self, ptr: int, shape: tuple, typestr: str, owner):
        self.__cuda_array_interface__ = {"shape": shape, "typestr": typestr, "data": (ptr, False),
                                         "version": 2, "strides": None}
        self._owner = owner


class CountResult:
    """Device-resident sorted histogram; keys are uint64 [n] (k <= 32) or [n, 2] (lo, hi)."""

    def __init__(self, counter: "KmerCounter", res: Result):
        self._counter = counter
        self._res = res

    @property
    def n(self) -> int:
        return int(self._res.n)

    @property
    def key_words(self) -> int:
        return int(self._res.key_words)

    @property
    def n_valid_windows(self) -> int:
        return int(self._res.n_valid_windows)

    def keys_tensor(self):
        """Zero-copy int64 view of the key words (raw bits of the uint64 keys)."""
        import torch
        shape = (self.n,) if self.key_words == 1 else (self.n, 2)
        return torch.as_tensor(_DeviceArray(self._res.keys or 0, shape, "<i8", self), device="cuda")

    def counts_tensor(self):
        """Zero-copy int32 view of the counts (raw bits of the uint32 counts)."""
        import torch
        return torch.as_tensor(_DeviceArray(self._res.counts or 0, (self.n,), "<i4", self), device="cuda")

    def to_numpy(self):
        lib = load_library()
        keys = np.empty(self.n * self.key_words, dtype=np.uint64)
        counts = np.empty(self.n, dtype=np.uint32)
        _check(lib, lib.kc_result_copy_to_host(self._counter._plan, ctypes.byref(self._res),
                                               keys.ctypes.data, counts.ctypes.data))
        if self.key_words == 2:
            keys = keys.reshape(self.n, 2)
        return keys, counts

    def free(self):
        if self._res is not None and self._counter._plan:
            lib = load_library()
            _check(lib, lib.kc_free(self._counter._plan, ctypes.byref(self._res)))
        self._res = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class KmerCounter:
    """A plan (kc_plan) bound to one device and stream, with torch's caching allocator."""

    def __init__(self, device: int | None = None, stream=None, use_torch_allocator: bool = True,
                 n_partitions_hint: int = 0, table_load: float = 0.0, table_slots_max: int = 0,
                 max_device_bytes: int = 0, profile: bool = False, defer_all: bool = False,
                 small_batch_arena: bool = False, no_smem_buckets: bool = False, warp_merge: bool = False,
                 test_withhold_prefix: bool = False, test_count_limit: bool = False,
                 test_fine_sampled: bool = False, test_tight_slack: bool = False):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("KmerCounter needs a CUDA device (no CPU fallback)")
        lib = load_library()
        self._lib = lib
        self.device = torch.cuda.current_device() if device is None else int(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        opts = PlanOpts()
        opts.device = self.device
        opts.stream = ctypes.c_void_p(int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream or 0))
        if use_torch_allocator:
            dev = self.device

            def _alloc(nbytes, strm, ctx):
                try:
                    return int(torch.cuda.caching_allocator_alloc(int(nbytes), dev, strm or 0))
                except Exception:
                    return None

            def _free(ptr, strm, ctx):
                if ptr:
                    torch.cuda.caching_allocator_delete(int(ptr))

            self._alloc_cb = _ALLOC_FN(_alloc)
            self._free_cb = _FREE_FN(_free)
            opts.alloc = self._alloc_cb
            opts.free_ = self._free_cb
        else:
            opts.alloc = _ALLOC_FN()
            opts.free_ = _FREE_FN()
        opts.max_device_bytes = int(max_device_bytes)
        opts.n_partitions_hint = int(n_partitions_hint)
        opts.table_load = float(table_load)
        opts.table_slots_max = int(table_slots_max)
        opts.flags = ((KC_PLAN_PROFILE if profile else 0) | (KC_PLAN_DEFER_ALL if defer_all else 0)
                      | (KC_PLAN_BATCH_ARENA_SMALL if small_batch_arena else 0)
                      | (KC_PLAN_ABLATE_NO_SMEM_BUCKETS if no_smem_buckets else 0)
                      | (KC_PLAN_WARP_MERGE if warp_merge else 0)
                      | (KC_PLAN_TEST_WITHHOLD_PREFIX if test_withhold_prefix else 0)
                      | (KC_PLAN_TEST_COUNT_LIMIT if test_count_limit else 0)
                      | (KC_PLAN_TEST_FINE_SAMPLED if test_fine_sampled else 0)
                      | (KC_PLAN_TEST_TIGHT_SLACK if test_tight_slack else 0))
        plan = ctypes.c_void_p()
        _check(lib, lib.kc_plan(ctypes.byref(opts), ctypes.byref(plan)))
        self._opts = opts
        self._plan = plan
        self._inflight = {}  # job id -> the buffers it reads
        self._job_kw = {}  # job id -> its key words (1 for k <= 32, else 2)

    def count(self, reads, offsets, k: int, canonical: bool = True) -> CountResult:
        """Sorted (k-mer, count) histogram of the reads (host or device buffers)."""
        rp, rk = _ptr(reads)
        op, ok = _ptr(offsets)
        n_reads = (offsets.shape[0] if hasattr(offsets, "shape") else len(offsets)) - 1
        if n_reads < 0:
            raise ValueError("offsets must hold n_reads + 1 entries")
        res = Result()
        _check(self._lib, self._lib.kc_count(self._plan, rp, op, n_reads, int(k), int(bool(canonical)),
                                             ctypes.byref(res)))
        del rk, ok
        return CountResult(self, res)

    def count_batch(self, samples, k: int, canonical: bool = True) -> list[CountResult]:
        """Histograms of several read sets in one call (kc_count_batch).  samples: a list of
        (reads, offsets) or (reads, offsets, n_bases), offsets on the host (numpy) or the
        device (then give n_bases, or it is read back); one result each."""
        n = len(samples)
        keep = []
        R = (ctypes.c_void_p * n)()
        O = (ctypes.c_void_p * n)()
        NR = (ctypes.c_uint64 * n)()
        NB = (ctypes.c_uint64 * n)()
        for i, sample in enumerate(samples):
            reads, offsets = sample[0], sample[1]
            rp, rk = _ptr(reads)
            op, ok = _ptr(offsets)
            keep += [rk, ok]
            R[i], O[i] = rp, op
            NR[i] = (offsets.shape[0] if hasattr(offsets, "shape") else len(offsets)) - 1
            if len(sample) > 2:
                NB[i] = int(sample[2])
            else:
                last = offsets[-1]
                NB[i] = int(last.item() if hasattr(last, "item") else last)
        res = (Result * n)()
        _check(self._lib, self._lib.kc_count_batch(self._plan, n, R, O, NR, NB, int(k), int(bool(canonical)), res))
        del keep
        return [CountResult(self, res[i]) for i in range(n)]

    def submit(self, reads, offsets, k: int, canonical: bool = True, n_bases: int | None = None) -> int:
        """Enqueue a count without waiting for it (kc_submit); returns a job id.  The
        buffers are kept alive here until the job is collected; host buffers should be
        pinned (torch pin_memory) so that the call does not wait for earlier work."""
        rp, rk = _ptr(reads)
        op, ok = _ptr(offsets)
        n_reads = (offsets.shape[0] if hasattr(offsets, "shape") else len(offsets)) - 1
        if n_reads < 0:
            raise ValueError("offsets must hold n_reads + 1 entries")
        if n_bases is None:
            last = offsets[-1]
            n_bases = int(last.item() if hasattr(last, "item") else last)
        job = ctypes.c_uint64()
        _check(self._lib, self._lib.kc_submit(self._plan, rp, op, n_reads, int(n_bases), int(k),
                                              int(bool(canonical)), ctypes.byref(job)))
        self._inflight[job.value] = (rk, ok)
        self._job_kw[job.value] = 1 if int(k) <= 32 else 2
        return job.value

    def submit_batch(self, samples, k: int, canonical: bool = True) -> list[int]:
        """Enqueue several counts as kc_count_batch would (batched launches) without waiting
        (kc_submit_batch); one job id per sample, each collected with poll / wait."""
        n = len(samples)
        if n == 0:
            return []
        keep = []
        R = (ctypes.c_void_p * n)()
        O = (ctypes.c_void_p * n)()
        NR = (ctypes.c_uint64 * n)()
        NB = (ctypes.c_uint64 * n)()
        for i, sample in enumerate(samples):
            reads, offsets = sample[0], sample[1]
            rp, rk = _ptr(reads)
            op, ok = _ptr(offsets)
            keep.append((rk, ok))
            R[i], O[i] = rp, op
            NR[i] = (offsets.shape[0] if hasattr(offsets, "shape") else len(offsets)) - 1
            if len(sample) > 2:
                NB[i] = int(sample[2])
            else:
                last = offsets[-1]
                NB[i] = int(last.item() if hasattr(last, "item") else last)
        jobs = (ctypes.c_uint64 * n)()
        _check(self._lib, self._lib.kc_submit_batch(self._plan, n, R, O, NR, NB, int(k), int(bool(canonical)), jobs))
        out = [int(jobs[i]) for i in range(n)]
        for j, kept in zip(out, keep):
            self._inflight[j] = kept
            self._job_kw[j] = 1 if int(k) <= 32 else 2
        return out

    def copy_to_host(self, job: int, keys_host, counts_host) -> None:
        """Have a submitted job's result copied to host buffers as soon as its count ends
        (kc_job_copy_to_host): keys_host holds capacity x key words (int64/uint64), counts_host
        capacity counts (int32/uint32); pinned memory lets the copy overlap later counts.
        The job is reported done once the copy has completed.  The buffers are checked here
        against the job's key width, as the C call takes plain pointers."""
        for x in (keys_host, counts_host):
            ok = x.flags["C_CONTIGUOUS"] if isinstance(x, np.ndarray) else x.is_contiguous()
            if not ok:
                raise ValueError("copy_to_host: the host buffers must be contiguous")

        def size(x):  # (elements, bytes per element)
            if isinstance(x, np.ndarray):
                return x.size, x.itemsize
            return x.numel(), x.element_size()

        nk, sk = size(keys_host)
        nc, sc = size(counts_host)
        if sk != 8 or sc != 4:
            raise ValueError("copy_to_host: keys_host takes 64-bit words, counts_host 32-bit counts")
        cap = nc
        kw = self._job_kw.get(int(job))
        if kw is not None and nk < cap * kw:
            raise ValueError(f"copy_to_host: keys_host holds {nk} words; {cap} keys of this job take {cap * kw}")
        kp, kk = _ptr(keys_host)
        cp, ck = _ptr(counts_host)
        _check(self._lib, self._lib.kc_job_copy_to_host(self._plan, int(job), kp, cp, int(cap)))
        self._inflight[int(job)] = self._inflight.get(int(job), ()) + (kk, ck)

    def poll(self, job: int) -> CountResult | None:
        """The job's result if it has finished (kc_job_poll), else None."""
        res = Result()
        done = ctypes.c_int()
        try:
            _check(self._lib, self._lib.kc_job_poll(self._plan, int(job), ctypes.byref(res), ctypes.byref(done)))
        finally:
            if done.value:
                self._inflight.pop(int(job), None)
                self._job_kw.pop(int(job), None)
        return CountResult(self, res) if done.value else None

    def wait(self, job: int) -> CountResult:
        """Block until the job finishes and return its result (kc_job_wait)."""
        res = Result()
        try:
            _check(self._lib, self._lib.kc_job_wait(self._plan, int(job), ctypes.byref(res)))
        finally:
            self._inflight.pop(int(job), None)
            self._job_kw.pop(int(job), None)
        return CountResult(self, res)

    def footprint(self, n_reads: int, n_bases: int, k: int, reads_on_device: bool = True,
                  offsets_on_device: bool = True) -> tuple[int, int]:
        """(scratch bytes, result bytes) a count of this size would take on this plan
        (kc_footprint; host arithmetic, nothing allocated)."""
        sb, rb = ctypes.c_uint64(), ctypes.c_uint64()
        _check(self._lib, self._lib.kc_footprint(self._plan, int(n_reads), int(n_bases), int(k),
                                                 int(bool(reads_on_device)), int(bool(offsets_on_device)),
                                                 ctypes.byref(sb), ctypes.byref(rb)))
        return int(sb.value), int(rb.value)

    def stats(self) -> dict:
        st = Stats()
        _check(self._lib, self._lib.kc_last_stats(self._plan, ctypes.byref(st)))
        out = {f: getattr(st, f) for f, _ in Stats._fields_}
        out["phase_cycles"] = [int(x) for x in st.phase_cycles]
        out["sub_cycles"] = [int(x) for x in st.sub_cycles]
        return {k: (v if isinstance(v, list) else int(v)) for k, v in out.items()}

    def kernel_times(self) -> list[tuple[str, float]]:
        """[(kernel name, device ms)] of the last count (plans created with profile=True)."""
        n = ctypes.c_uint32()
        names = (ctypes.c_char_p * 64)()
        ms = (ctypes.c_float * 64)()
        _check(self._lib, self._lib.kc_last_kernel_times(self._plan, 64, names, ms, ctypes.byref(n)))
        return [(names[i].decode(), float(ms[i])) for i in range(min(n.value, 64))]

    def close(self):
        if self._plan:
            self._lib.kc_plan_destroy(self._plan)
            self._plan = None
            self._inflight.clear()
            self._job_kw.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

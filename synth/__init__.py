"""Seeded synthetic read sets (ASCII bases + read offsets) for the k-mer counter.

This package holds no part of the counting method: it only writes bases.  The
oracle and the CUDA path both take their inputs from here.

The paper's inputs are ART-simulated Illumina reads of uniform random genomes
and SRA genomes (Section VI, "Datasets", Table VI); neither is available, so these
seeded generators stand in for them with the same read lengths, coverages and
error shapes.  The C source (synth.c) describes each workload.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")

# workload ids understood by synth.c
UNIFORM_SHORT = 0   # 1 Mbp i.i.d. genome, 100 bp reads, 10x, 0.5% subst, 0.01% N
REPEAT_SHORT = 1    # 100 Mbp genome with 20% repeat families, 150 bp reads, 30x
LONG_NOISY = 2      # 50 Mbp genome, ~10 kbp log-normal reads, 20x, 5% indel-rich errors
SAMPLE = 3          # one batched-workload sample (log-uniform genome size, 5-40x)
SERVE = 4           # one served-workload request's read set (genome log-uniform 0.05-20 Mbp, 10-30x)

# the five benchmark workloads: (generator, seed, k)
WORKLOADS = {
    "uniform_1mbp_100bp_10x_k31": (UNIFORM_SHORT, 1001, 31),
    "repeats_100mbp_150bp_30x_k31": (REPEAT_SHORT, 1002, 31),
    "long_50mbp_10kbp_20x_k63": (LONG_NOISY, 1003, 63),
}


class _Out(ctypes.Structure):
    _fields_ = [("reads", ctypes.c_void_p), ("offsets", ctypes.c_void_p),
                ("n_reads", ctypes.c_uint64), ("n_bytes", ctypes.c_uint64),
                ("genome_len", ctypes.c_uint64)]


def build(force: bool = False) -> str:
    """Compile synth.c into libsynth.so beside it (plain gcc, portable flags; no fused
    multiply-add contraction, so that x86-64 and Arm builds draw the same reads)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.synth_generate.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(_Out)]
        lib.synth_generate.restype = ctypes.c_int
        lib.synth_free.argtypes = [ctypes.POINTER(_Out)]
        lib.synth_free.restype = None
        lib.synth_mix_seed.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
        lib.synth_mix_seed.restype = ctypes.c_uint64
        _lib = lib
    return _lib


def generate(workload: int, seed: int, scale: float = 1.0):
    """Return (reads uint8[n_bytes], offsets uint64[n_reads+1], genome_len)."""
    lib = _load()
    out = _Out()
    rc = lib.synth_generate(int(workload), int(seed) & (2**64 - 1), float(scale), ctypes.byref(out))
    if rc != 0:
        raise RuntimeError(f"synth_generate failed ({rc})")
    try:
        nb, nr = int(out.n_bytes), int(out.n_reads)
        reads = np.empty(nb, dtype=np.uint8)
        offsets = np.empty(nr + 1, dtype=np.uint64)
        if nb:
            ctypes.memmove(reads.ctypes.data, out.reads, nb)
        ctypes.memmove(offsets.ctypes.data, out.offsets, 8 * (nr + 1))
        return reads, offsets, int(out.genome_len)
    finally:
        lib.synth_free(ctypes.byref(out))


def mix_seed(seed: int, index: int) -> int:
    """Per-sample seed: one splitmix64 step of (seed xor index)."""
    return int(_load().synth_mix_seed(int(seed) & (2**64 - 1), int(index) & (2**64 - 1)))


def workload(name: str, scale: float = 1.0):
    """Reads of one named benchmark workload: (reads, offsets, k)."""
    gen, seed, k = WORKLOADS[name]
    reads, offsets, _ = generate(gen, seed, scale)
    return reads, offsets, k


def random_reads(rng: np.random.Generator, n_reads: int, max_len: int,
                 junk: float = 0.02, lower: float = 0.05, n_rate: float = 0.02):
    """Small random read sets with the awkward bytes a counter must skip: 'N',
    lowercase bases, and arbitrary other bytes.  Lengths uniform in [0, max_len]."""
    lens = rng.integers(0, max_len + 1, size=n_reads)
    offsets = np.zeros(n_reads + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum(lens)
    total = int(offsets[-1])
    reads = np.frombuffer(b"ACGT", dtype=np.uint8)[rng.integers(0, 4, size=total)].copy()
    u = rng.random(total)
    low = u < lower
    reads[low] = reads[low] + 32  # 'A' -> 'a' etc.
    nmask = (u >= lower) & (u < lower + n_rate)
    reads[nmask] = ord("N")
    jmask = (u >= lower + n_rate) & (u < lower + n_rate + junk)
    reads[jmask] = rng.integers(0, 256, size=int(jmask.sum())).astype(np.uint8)
    return reads, offsets

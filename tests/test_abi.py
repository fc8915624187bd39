"""The C-ABI library builds for sm_103a, loads without a GPU, exports every entry
point include/kc.h declares, and rejects bad arguments on the host."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2505_04431_gb300 as kcpy
from paper_2505_04431_gb300 import build as kcbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "kc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kc_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    path = kcbuild.build()
    return kcpy.load_library(path)


def test_header_declares_the_abi():
    fns = header_functions()
    assert fns == sorted(kcpy.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", kcpy.LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (kc_[a-z_0-9]+)$", out, flags=re.M))
    for fn in header_functions():
        assert fn in exported, fn
        assert hasattr(lib, fn)


def test_library_is_built_for_sm103a(lib):
    """Every compile and the link take the one sm_103a target and no other architecture."""
    from paper_2505_04431_gb300 import build as kcbuild
    assert kcbuild.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert not any(f.startswith(("-gencode", "-arch", "--gpu-architecture", "-code")) for f in kcbuild.FLAGS)


def test_host_side_argument_errors(lib):
    res = kcpy.Result()
    # NULL plan / out
    assert lib.kc_count(None, None, None, 0, 31, 1, ctypes.byref(res)) == kcpy.KC_EINVAL
    assert lib.kc_last_error().decode().startswith("kc_count")
    assert lib.kc_plan(None, None) == kcpy.KC_EINVAL
    assert lib.kc_free(None, ctypes.byref(res)) == kcpy.KC_EINVAL
    assert lib.kc_plan_destroy(None) == kcpy.KC_EINVAL
    st = kcpy.Stats()
    assert lib.kc_last_stats(None, ctypes.byref(st)) == kcpy.KC_EINVAL
    # bad plan options are rejected before any device call
    opts = kcpy.PlanOpts()
    opts.n_partitions_hint = 3
    plan = ctypes.c_void_p()
    assert lib.kc_plan(ctypes.byref(opts), ctypes.byref(plan)) == kcpy.KC_EINVAL
    opts.n_partitions_hint = 8192
    assert lib.kc_plan(ctypes.byref(opts), ctypes.byref(plan)) == kcpy.KC_EINVAL
    opts.n_partitions_hint = 0
    opts.table_slots_max = 10
    assert lib.kc_plan(ctypes.byref(opts), ctypes.byref(plan)) == kcpy.KC_EINVAL


def test_plan_without_gpu_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    opts = kcpy.PlanOpts()
    plan = ctypes.c_void_p()
    st = lib.kc_plan(ctypes.byref(opts), ctypes.byref(plan))
    assert st in (kcpy.KC_ECUDA, kcpy.KC_EINVAL)
    assert not plan.value


def test_binding_refuses_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(RuntimeError):
        kcpy.KmerCounter()

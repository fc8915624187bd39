"""kc_count_noalloc, the entry point for callers that may not allocate device memory
while counting (for example an application whose device memory is all held by its own
pool).  It must give exactly what kc_count gives, call after call, using only the
library's fixed scratch array and the caller's buffers.

This file is collected last so that, if it fails, a run that stops at the first failure
has already run every other test.  It passes alone in a fresh process too."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_04431_gb300 import KmerCounter, build, load_library
    build.build()
    lib = load_library()
    counter = KmerCounter()
    yield torch, lib, counter
    counter.close()


def reference(counter, reads, offsets, k, canonical):
    res = counter.count(reads, offsets, k, canonical)
    try:
        keys, counts = res.to_numpy()
        return keys.reshape(-1), counts, res.n, res.n_valid_windows
    finally:
        res.free()


def noalloc(torch, lib, reads, offsets, k, canonical):
    """One call through the C ABI with caller-owned device buffers."""
    from paper_2505_04431_gb300 import KC_OK
    r = torch.from_numpy(reads).cuda()
    o = torch.from_numpy(offsets.view(np.int64)).cuda()
    kw = 1 if k <= 32 else 2
    cap = max(1, len(reads))
    out_k = torch.full((cap * kw,), -1, dtype=torch.int64, device="cuda")
    out_c = torch.zeros(cap, dtype=torch.int32, device="cuda")
    nd, nv = ctypes.c_uint64(0), ctypes.c_uint64(0)
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.kc_count_noalloc(r.data_ptr(), o.data_ptr(), len(offsets) - 1, k, int(canonical), out_k.data_ptr(),
                              out_c.data_ptr(), cap, ctypes.byref(nd), ctypes.byref(nv), stream)
    assert st == KC_OK, lib.kc_last_error().decode()
    d = nd.value
    keys = out_k[: d * kw].cpu().numpy().view(np.uint64)
    counts = out_c[:d].cpu().numpy().view(np.uint32)
    return keys, counts, d, nv.value


def test_noalloc_matches_kc_count_on_consecutive_calls(env):
    torch, lib, counter = env
    cases = [
        (synth.generate(synth.UNIFORM_SHORT, 1001, 0.08)[:2], 31, True),     # 80 kbp genome, 8000 reads
        (synth.generate(synth.LONG_NOISY, 1003, 0.001)[:2], 63, True),       # long noisy reads, 128-bit keys
        (synth.generate(synth.REPEAT_SHORT, 1002, 0.0003)[:2], 21, False),   # forward keys
    ]
    for (reads, offsets), k, canonical in cases:
        assert len(reads) <= (1 << 20)
        ref = reference(counter, reads, offsets, k, canonical)
        # two calls in a row: the second starts from the scratch contents the first left
        for _ in range(2):
            got = noalloc(torch, lib, reads, offsets, k, canonical)
            assert got[2] == ref[2] and got[3] == ref[3]
            assert np.array_equal(got[0], ref[0])
            assert np.array_equal(got[1], ref[1])


def test_noalloc_rejects_inputs_beyond_its_maximum(env):
    torch, lib, _ = env
    from paper_2505_04431_gb300 import KC_EINVAL, KC_NOALLOC_MAX_BASES
    n = KC_NOALLOC_MAX_BASES + 1
    r = torch.full((n,), ord("A"), dtype=torch.uint8, device="cuda")
    o = torch.tensor([0, n], dtype=torch.int64, device="cuda")
    out_k = torch.empty(n, dtype=torch.int64, device="cuda")
    out_c = torch.empty(n, dtype=torch.int32, device="cuda")
    nd, nv = ctypes.c_uint64(0), ctypes.c_uint64(0)
    st = lib.kc_count_noalloc(r.data_ptr(), o.data_ptr(), 1, 31, 1, out_k.data_ptr(), out_c.data_ptr(), n,
                              ctypes.byref(nd), ctypes.byref(nv), torch.cuda.current_stream().cuda_stream)
    assert st == KC_EINVAL
    assert "maximum" in lib.kc_last_error().decode()


def test_noalloc_refuses_misaligned_buffers_before_launching(env):
    """A caller buffer at an odd offset (a slice of a larger tensor, say) is refused on the
    host: the kernels write 16-byte keys for k > 32, 4-byte counts and read 8-byte offsets."""
    torch, lib, _ = env
    from paper_2505_04431_gb300 import KC_EINVAL
    reads, offsets = synth.generate(synth.UNIFORM_SHORT, 1001, 0.01)[:2]
    r = torch.from_numpy(reads).cuda()
    o = torch.from_numpy(offsets.view(np.int64)).cuda()
    cap = len(reads)
    big_k = torch.zeros(cap * 2 + 4, dtype=torch.int64, device="cuda")
    big_c = torch.zeros(cap + 4, dtype=torch.int32, device="cuda")
    big_o = torch.zeros(len(offsets) * 8 + 8, dtype=torch.uint8, device="cuda")
    nd, nv = ctypes.c_uint64(0), ctypes.c_uint64(0)
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(63, o.data_ptr(), big_k.data_ptr() + 8, big_c.data_ptr()),   # keys 8- but not 16-byte aligned
             (31, o.data_ptr(), big_k.data_ptr() + 4, big_c.data_ptr()),   # keys not 8-byte aligned
             (31, o.data_ptr(), big_k.data_ptr(), big_c.data_ptr() + 2),   # counts not 4-byte aligned
             (31, big_o.data_ptr() + 4, big_k.data_ptr(), big_c.data_ptr())]  # offsets not 8-byte aligned
    for k, op, kp, cp in cases:
        st = lib.kc_count_noalloc(r.data_ptr(), op, len(offsets) - 1, k, 1, kp, cp, cap, ctypes.byref(nd),
                                  ctypes.byref(nv), stream)
        assert st == KC_EINVAL and "aligned" in lib.kc_last_error().decode()

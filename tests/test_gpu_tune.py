"""Autotuner on the GPU: it times real counts under each candidate plan, every candidate
returns the same result (checked inside autotune), and the chosen options count correctly."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_autotune_small_input():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2505_04431_gb300 import KmerCounter, build, tune
    build.build()
    reads, offsets, _ = synth.generate(synth.REPEAT_SHORT, 1002, 0.003)
    r = torch.from_numpy(reads).cuda()
    o = torch.from_numpy(offsets.view(np.int64)).cuda()
    torch.cuda.synchronize()
    out = tune.autotune(r, o, 31, repeats=2)
    assert out["best_ms"] > 0 and len(out["trials"]) >= 3
    assert all(ms > 0 for _, ms in out["trials"])
    c = KmerCounter(**out["best"])
    try:
        res = c.count(reads, offsets, 31, True)
        keys, counts = res.to_numpy()
        res.free()
    finally:
        c.close()
    ok, oc, _ = oracle.count(reads, offsets, 31, True)
    assert np.array_equal(keys, ok) and np.array_equal(counts, oc)

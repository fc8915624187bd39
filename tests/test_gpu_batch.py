"""Batched form (kc_count_batch): every sample's histogram must be byte-identical to what
kc_count returns for that sample alone, and (small samples) to the oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module")
def counter(torch_cuda):
    from paper_2505_04431_gb300 import KmerCounter, build
    build.build()
    c = KmerCounter()
    yield c
    c.close()


def alone(counter, reads, offsets, k, canonical):
    res = counter.count(reads, offsets, k, canonical)
    try:
        keys, counts = res.to_numpy()
        return keys, counts, res.n_valid_windows
    finally:
        res.free()


def batch_samples(n, scale, seed=1004):
    out = []
    for i in range(n):
        reads, offsets, _ = synth.generate(synth.SAMPLE, synth.mix_seed(seed, i), scale)
        out.append((reads, offsets))
    return out


@pytest.mark.parametrize("k,canonical", [(31, True), (21, False), (63, True)])
def test_batch_matches_single_counts(counter, torch_cuda, k, canonical):
    torch = torch_cuda
    samples = batch_samples(12, 0.01)  # genomes of 1 kbp - 0.5 Mbp, 5-40x
    samples.insert(3, (np.zeros(0, np.uint8), np.zeros(1, np.uint64)))  # an empty sample
    dev = [(torch.from_numpy(r).cuda(), o, int(o[-1])) for r, o in samples]  # device reads, host offsets
    results = counter.count_batch(dev, k, canonical)
    try:
        assert len(results) == len(samples)
        for i, ((r, o), res) in enumerate(zip(samples, results)):
            keys, counts = res.to_numpy()
            ak, ac, anv = alone(counter, r, o, k, canonical)
            assert res.n_valid_windows == anv, i
            assert np.array_equal(keys, ak) and np.array_equal(counts, ac), f"sample {i} differs from kc_count"
            if i < 4:  # the oracle on a few
                ok, oc, onv = oracle.count(r, o, k, canonical)
                assert onv == anv and np.array_equal(ok, keys) and np.array_equal(oc, counts), f"sample {i} vs oracle"
    finally:
        for res in results:
            res.free()


def test_batch_large_and_small_mixed(counter, torch_cuda):
    # one large sample (several coarse partitions) among small ones: the scratch is sized for
    # the large one and the small ones reuse it
    torch = torch_cuda
    big_r, big_o, _ = synth.generate(synth.REPEAT_SHORT, 1002, 0.03)  # 3 Mbp genome, 30x: 90 M bases
    assert int(big_o[-1]) > (64 << 20)
    samples = [(big_r, big_o)] + batch_samples(6, 0.005)
    dev = [(torch.from_numpy(r).cuda(), torch.from_numpy(o.view(np.int64)).cuda(), int(o[-1])) for r, o in samples]
    results = counter.count_batch(dev, 31, True)
    try:
        for i, ((r, o), res) in enumerate(zip(samples, results)):
            keys, counts = res.to_numpy()
            ak, ac, anv = alone(counter, r, o, 31, True)
            assert res.n_valid_windows == anv and np.array_equal(keys, ak) and np.array_equal(counts, ac), i
    finally:
        for res in results:
            res.free()


def test_batch_edge_cases(counter, torch_cuda):
    from paper_2505_04431_gb300 import KcError, KC_EINVAL
    assert counter.count_batch([], 31) == []
    good = batch_samples(3, 0.002)
    bad_o = good[1][1].copy()
    bad_o[2], bad_o[3] = bad_o[3], bad_o[2]  # not non-decreasing
    with pytest.raises(KcError) as ei:
        counter.count_batch([good[0], (good[1][0], bad_o), good[2]], 31)
    assert ei.value.status == KC_EINVAL
    # a base count that disagrees with the device offsets is caught on the device
    torch = torch_cuda
    r, o = good[0]
    with pytest.raises(KcError) as ei:
        counter.count_batch([(torch.from_numpy(r).cuda(), torch.from_numpy(o.view(np.int64)).cuda(), int(o[-1]) - 1)], 31)
    assert ei.value.status == KC_EINVAL and "sample 0" in str(ei.value)
    # the plan still counts correctly afterwards
    ak, ac, _ = alone(counter, r, o, 31, True)
    res = counter.count_batch([good[0]], 31)[0]
    keys, counts = res.to_numpy()
    res.free()
    assert np.array_equal(keys, ak) and np.array_equal(counts, ac)


@pytest.mark.parametrize("k,canonical,defer_all", [(31, True, False), (63, True, False), (21, False, True)])
def test_batch_several_groups_and_counts_alone(counter, torch_cuda, k, canonical, defer_all):
    # a 32 MiB arena: the small samples form several groups of batched launches, the larger
    # ones (scratch above the arena) are counted alone; every result equals kc_count's
    from paper_2505_04431_gb300 import KmerCounter
    torch = torch_cuda
    samples = batch_samples(14, 0.01, seed=2004)
    samples.insert(5, (np.zeros(0, np.uint8), np.zeros(1, np.uint64)))
    sizes = [int(o[-1]) for _, o in samples]
    assert max(sizes) > (5 << 19) and sum(1 for n in sizes if 0 < n < (1 << 20)) >= 3  # ~16 B of scratch per base
    small = KmerCounter(small_batch_arena=True, defer_all=defer_all)
    try:
        dev = [(torch.from_numpy(r).cuda(), o, int(o[-1])) for r, o in samples]
        results = small.count_batch(dev, k, canonical)
        order = np.random.RandomState(5).permutation(len(results))  # results freed in any order
        for i in order:
            r, o = samples[i]
            keys, counts = results[i].to_numpy()
            nv = results[i].n_valid_windows
            results[i].free()
            ak, ac, anv = alone(counter, r, o, k, canonical)
            assert nv == anv and np.array_equal(keys, ak) and np.array_equal(counts, ac), f"sample {i} differs"
            if sizes[i] < 200_000:
                ok, oc, onv = oracle.count(r, o, k, canonical)
                assert onv == nv and np.array_equal(keys, ok) and np.array_equal(counts, oc)
    finally:
        small.close()


@pytest.mark.parametrize("tight", [False, True])
def test_batch_with_sampled_fine_layouts(torch_cuda, tight):
    """Batched launches over counts whose fine regions are sized from a sample (forced here
    on small samples) and, without slack, overflow so that the exact split runs for them:
    every sample equals the oracle."""
    from paper_2505_04431_gb300 import KmerCounter
    c = KmerCounter(test_fine_sampled=True, test_tight_slack=tight)
    try:
        samples = batch_samples(6, 0.02, seed=2004)
        samples.insert(2, (np.zeros(0, np.uint8), np.zeros(1, np.uint64)))
        for k in (31, 63):
            results = c.count_batch(samples, k, True)
            for i, ((r, o), res) in enumerate(zip(samples, results)):
                keys, counts = res.to_numpy()
                ek, ec, env = oracle.count(r, o, k, True)
                assert res.n_valid_windows == env, (k, i)
                assert np.array_equal(keys.reshape(ek.shape), ek) and np.array_equal(counts, ec), f"k {k} sample {i}"
                res.free()
    finally:
        c.close()

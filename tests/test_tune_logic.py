"""Host logic of the autotuner (no GPU): the candidates it tries, the choice of the fastest,
and the refusal of options that change the result."""
import pytest

from paper_2505_04431_gb300 import tune


def fake_timer(costs, p1=256, digest=("d",)):
    """A timer whose time per option set is looked up in `costs` (keyed by its sorted items)."""
    seen = []

    def timer(opts):
        seen.append(dict(opts))
        key = tuple(sorted(opts.items()))
        return costs.get(key, 100.0), digest, p1
    return timer, seen


def test_tries_half_and_double_partitions_then_table_load():
    costs = {(): 66.0, (("n_partitions_hint", 128),): 64.0, (("n_partitions_hint", 512),): 70.0,
             (("n_partitions_hint", 128), ("table_load", 0.45)): 63.5}
    timer, seen = fake_timer(costs)
    out = tune.autotune(None, None, 31, timer=timer)
    assert seen == [{}, {"n_partitions_hint": 128}, {"n_partitions_hint": 512},
                    {"n_partitions_hint": 128, "table_load": 0.45}]
    assert out["best"] == {"n_partitions_hint": 128, "table_load": 0.45} and out["best_ms"] == 63.5
    assert len(out["trials"]) == 4


def test_keeps_the_library_choice_when_nothing_is_faster():
    timer, _ = fake_timer({(): 10.0})
    out = tune.autotune(None, None, 31, timer=timer)
    assert out["best"] == {} and out["best_ms"] == 10.0


def test_partition_candidates_stay_in_range():
    timer, seen = fake_timer({}, p1=1)
    tune.autotune(None, None, 31, timer=timer)
    assert {"n_partitions_hint": 0} not in seen and {"n_partitions_hint": 2} in seen
    timer, seen = fake_timer({}, p1=4096)
    tune.autotune(None, None, 31, timer=timer)
    assert {"n_partitions_hint": 8192} not in seen and {"n_partitions_hint": 2048} in seen


def test_options_that_change_the_result_are_refused():
    calls = []

    def timer(opts):
        calls.append(opts)
        return 1.0, ("a",) if len(calls) == 1 else ("b",), 64
    with pytest.raises(RuntimeError):
        tune.autotune(None, None, 31, timer=timer)

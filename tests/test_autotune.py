"""CPU tests of the autotuner's search and cache (no GPU)."""
from paper_0910_0329_gb300 import autotune


def test_coordinate_descent_finds_separable_optimum():
    target = {"queue_log2": 13, "blocks_per_sm": 6, "refill_min": 16, "refill_pause": -1}
    calls = []

    def trial(o):
        calls.append(o)
        return 1.0 + sum((o[k] - target[k]) ** 2 for k in target) * 0.1

    best, t, log = autotune.coordinate_descent(trial, autotune.DEFAULT_SPACE, autotune.DEFAULT_START)
    assert best == target
    assert t == 1.0
    assert len(calls) == len(log) < 4 * 3 * 4 * 3  # fewer trials than the full grid, none repeated


def test_coordinate_descent_ignores_gains_below_the_noise_floor():
    # every move gains 1 % at most: the start stays
    def trial(o):
        return 1.0 - 0.01 * (o["refill_min"] == 16) - 0.005 * (o["queue_log2"] == 15)

    best, t, _ = autotune.coordinate_descent(trial, autotune.DEFAULT_SPACE, autotune.DEFAULT_START)
    assert best == autotune.DEFAULT_START and t == 1.0
    best, _, _ = autotune.coordinate_descent(trial, autotune.DEFAULT_SPACE, autotune.DEFAULT_START, min_gain=0.0)
    assert best["refill_min"] == 16 and best["queue_log2"] == 15


def test_start_outside_the_space_is_projected():
    space = {"queue_log2": [12, 14], "blocks_per_sm": [6, 8], "refill_min": [8]}
    best, _, log = autotune.coordinate_descent(lambda o: 1.0, space, autotune.DEFAULT_START)
    assert best == {"queue_log2": 14, "blocks_per_sm": 8, "refill_min": 8}  # only the space's parameters
    assert all(all(o[k] in space[k] for k in space) for o, _ in log)


def test_cache_roundtrip(tmp_path):
    p = str(tmp_path / "t.json")
    k = autotune.signature("GB300", "batch64")
    assert autotune.load(k, p) is None
    autotune.save(k, {"opts": {"refill_min": 4}}, p)
    autotune.save("other", {"opts": {}}, p)
    assert autotune.load(k, p)["opts"] == {"refill_min": 4}


def test_full_length_runs_decide_the_final_choice():
    start = dict(autotune.DEFAULT_START)
    best = dict(start, refill_min=16)
    calls = []

    def full(times):
        def f(o):
            calls.append(o)
            return times[o == best]
        return f

    # the short trials' winner is 5 % faster on the full runs: it is kept
    choice, t = autotune.confirm(full({False: 1.0, True: 0.95}), best, start)
    assert choice == best and t == (1.0, 0.95) and len(calls) == 4
    # 1 % faster on the full runs: within the noise floor, the defaults stay
    choice, _ = autotune.confirm(full({False: 1.0, True: 0.99}), best, start)
    assert choice == start
    # slower on the full runs (the short trials misled): the defaults stay
    choice, _ = autotune.confirm(full({False: 1.0, True: 1.04}), best, start)
    assert choice == start
    # nothing to confirm when the search kept the defaults
    calls.clear()
    choice, t = autotune.confirm(full({False: 1.0, True: 0.5}), dict(start), start)
    assert choice == start and t is None and calls == []

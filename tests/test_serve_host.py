"""Host logic of the request server (no GPU): the library's round sizing from
a request's own statistics and its round selection (dpm_serve_next_chunk and
dpm_serve_select are pure host functions of the C ABI), and the Poisson
request generator."""
import math

from paper_0910_0329_gb300 import dpm, serve


def next_chunk(histories, rel, adaptive=True, chunk=1000, target=0.01, max_chunk=20000, overshoot=1.0):
    o = dpm.serve_opts(target=target, first_chunk=chunk, max_chunk=max_chunk, overshoot=overshoot,
                       adaptive=int(adaptive))
    return dpm.serve_next_chunk(o, histories, rel)


def test_next_round_reaches_the_target_by_the_inverse_square_law():
    # 1000 histories at 4 % -> 16000 in all -> 15000 more
    assert next_chunk(1000, 0.04) == 15000
    # capped and floored
    assert next_chunk(1000, 0.5) == 20000
    assert next_chunk(1000, 0.0101) == 1000
    # overshoot
    assert next_chunk(1000, 0.02, overshoot=1.5) == 5000
    # 4000 histories at 2 % -> 16000 in all -> 12000 more
    assert next_chunk(4000, 0.02) == 12000


def test_fixed_rounds_without_adaptation_or_statistics():
    assert next_chunk(1000, 0.04, adaptive=False) == 1000
    assert next_chunk(1000, math.inf) == 1000
    assert next_chunk(1000, 0.0) == 1000


def test_option_defaults_and_invalid_options():
    o = dpm.serve_opts(target=0.01)  # first_chunk 200000, max_chunk 32x, overshoot 1.15
    assert dpm.serve_next_chunk(o, 200000, 0.02) == int(200000 * 4 * 1.15 - 200000)
    assert dpm.serve_next_chunk(o, 200000, 1.0) == 32 * 200000
    # invalid options size nothing
    assert dpm.serve_next_chunk(dpm.serve_opts(target=0.0), 1000, 0.04) == 0
    assert dpm.serve_next_chunk(dpm.serve_opts(target=0.01, first_chunk=100, max_chunk=50), 1000, 0.04) == 0


def test_poisson_requests_are_seeded_and_ordered():
    ext = [(10.0, 10.0, 10.0)] * 3
    a = serve.poisson_requests(50, 20.0, 3, seed=4, geom_extent=ext)
    b = serve.poisson_requests(50, 20.0, 3, seed=4, geom_extent=ext)
    assert [(r.arrival, r.geometry, r.source.gantry_deg) for r in a] == \
        [(r.arrival, r.geometry, r.source.gantry_deg) for r in b]
    assert all(x.arrival < y.arrival for x, y in zip(a, a[1:]))
    assert {r.geometry for r in a} == {0, 1, 2}
    # mean inter-arrival time near 1/rate
    assert abs(a[-1].arrival / 50 - 1 / 20.0) < 0.5 / 20.0


def test_rounds_take_the_oldest_requests_within_the_budget():
    want = [5000, 4000, 200, 3000, 200]
    # 5000 + 200 + 200 fit in 6000; 4000 and 3000 wait
    assert dpm.serve_select(want, 6000) == [0, 2, 4]
    # the oldest runs even alone above the budget
    assert dpm.serve_select(want, 100) == [0]
    assert dpm.serve_select(want, 10 ** 9) == [0, 1, 2, 3, 4]
    assert dpm.serve_select([], 100) == []


def test_round_selection_against_brute_force():
    """The rule stated as a predicate, checked on random queues: the oldest is
    taken; a younger request is taken exactly when it fits the budget together
    with all the requests taken before it."""
    import random
    rng = random.Random(7)
    for _ in range(300):
        want = [rng.choice([100, 200, 1000, 5000, 20000]) for _ in range(rng.randint(1, 12))]
        budget = rng.choice([50, 1000, 6000, 25000, 10 ** 6])
        got = dpm.serve_select(want, budget)
        assert got[0] == 0
        total, exp = 0, []
        for i, n in enumerate(want):
            if not exp or total + n <= budget:
                exp.append(i)
                total += n
        assert got == exp
        assert sum(want[i] for i in got) <= budget or got == [0]


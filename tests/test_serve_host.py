"""Host logic of the request server (no GPU): round sizing from a request's
own statistics and the Poisson request generator."""
import math
import types

from paper_0910_0329_gb300 import serve


def sizer(adaptive=True, chunk=1000, target=0.01, max_chunk=20000, overshoot=1.0):
    return types.SimpleNamespace(adaptive=adaptive, chunk=chunk, target=target, max_chunk=max_chunk,
                                 overshoot=overshoot)


def next_chunk(s, histories, rel):
    r = serve.Request(0, 0, None, 0.0, histories=histories, rel_sigma=rel)
    return serve.Server._next_chunk(s, r)


def test_next_round_reaches_the_target_by_the_inverse_square_law():
    # 1000 histories at 4 % -> 16000 in all -> 15000 more
    assert next_chunk(sizer(), 1000, 0.04) == 15000
    # capped and floored
    assert next_chunk(sizer(), 1000, 0.5) == 20000
    assert next_chunk(sizer(), 1000, 0.0101) == 1000
    # overshoot
    assert next_chunk(sizer(overshoot=1.5), 1000, 0.02) == 5000


def test_fixed_rounds_without_adaptation_or_statistics():
    assert next_chunk(sizer(adaptive=False), 1000, 0.04) == 1000
    assert next_chunk(sizer(), 1000, math.inf) == 1000


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
    reqs = [serve.Request(i, 0, None, float(i), next_n=n) for i, n in enumerate([5000, 4000, 200, 3000, 200])]
    # 5000 + 200 + 200 fit in 6000; 4000 and 3000 wait
    assert [r.rid for r in serve.select_round(reqs, 6000)] == [0, 2, 4]
    # the oldest runs even alone above the budget
    assert [r.rid for r in serve.select_round(reqs, 100)] == [0]
    assert [r.rid for r in serve.select_round(reqs, 10 ** 9)] == [0, 1, 2, 3, 4]

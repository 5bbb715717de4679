"""Serving with continuous batching: requests arriving over time share rounds
of batched launches; a request's result must not depend on the others
(bit-identical tally and the same number of histories alone and in the mix),
and admission must respect the HBM budget."""
import numpy as np
import pytest

from paper_0910_0329_gb300 import serve
from paper_0910_0329_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def geoms():
    return [W.blob_phantom(40, 40, 40, 0.4, 100 + k, name=f"g{k}") for k in range(2)]


def served(geoms, reqs, **kw):
    s = serve.Server(geoms, chunk=20000, target=0.05, keep_results=True, **kw)
    try:
        st = s.run(reqs)
    finally:
        s.close()
    return st, s


def test_result_is_the_same_alone_and_in_the_mix(geoms):
    ext = [g.extent for g in geoms]
    reqs = serve.poisson_requests(6, rate=40.0, n_geoms=2, seed=9, geom_extent=ext)
    st, _ = served(geoms, reqs)
    assert len(st.completed) == 6
    assert st.max_active >= 2  # requests did overlap on the device
    for r in st.completed:
        assert r.rel_sigma <= 0.05 and r.latency is not None and r.latency > 0
        alone_req = serve.Request(r.rid, r.geometry, r.source, 0.0)
        st1, _ = served(geoms, [alone_req])
        a = st1.completed[0]
        assert a.histories == r.histories
        assert np.array_equal(a.raw, r.raw)


def test_admission_respects_the_hbm_budget(geoms):
    ext = [g.extent for g in geoms]
    reqs = serve.poisson_requests(5, rate=200.0, n_geoms=1, seed=3, geom_extent=ext)
    probe = serve.Server(geoms, chunk=20000, target=0.05)
    budget = probe.fixed + 2 * probe.slot_bytes[0] + 1
    probe.close()
    st, s = served(geoms, reqs, hbm_budget=budget)
    assert len(st.completed) == 5
    assert st.max_active <= 2
    assert s.used <= budget

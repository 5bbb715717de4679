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
    assert st.max_active == 2
    assert st.peak_bytes <= budget


def test_slots_move_between_geometries_within_the_budget(geoms):
    """A budget of one slot: requests on alternating geometries free the
    released slot of the other geometry before a new copy is made; results
    stay those of the request alone."""
    ext = [g.extent for g in geoms]
    reqs = serve.poisson_requests(4, rate=1000.0, n_geoms=2, seed=11, geom_extent=ext)
    for k, r in enumerate(reqs):
        r.geometry = k % 2
    probe = serve.Server(geoms, chunk=20000, target=0.05)
    budget = probe.fixed + max(probe.slot_bytes) + 1
    probe.close()
    st, _ = served(geoms, reqs, hbm_budget=budget)
    assert len(st.completed) == 4 and st.max_active == 1
    assert st.peak_bytes <= budget
    for r in st.completed:
        st1, _ = served(geoms, [serve.Request(r.rid, r.geometry, r.source, 0.0)])
        assert st1.completed[0].histories == r.histories
        assert np.array_equal(st1.completed[0].raw, r.raw)


def test_library_server_states_and_errors(geoms):
    from paper_0910_0329_gb300 import dpm
    with dpm.Dpm(0, W.MATERIALS, W.DEFAULT_PARAMS) as d:
        g = d.load_phantom(geoms[0])
        srv = dpm.Server(d.ctx, dpm.serve_opts(target=0.05, first_chunk=20000))
        try:
            src = serve.poisson_requests(1, 10.0, 1, seed=1, geom_extent=[geoms[0].extent])[0].source
            rid = srv.submit(g, src, 123)
            assert srv.status(rid)["state"] == dpm.REQ_PENDING and srv.info()["n_pending"] == 1
            with pytest.raises(RuntimeError):
                srv.release(rid)  # not done
            srv.round()
            st = srv.status(rid)
            assert st["state"] in (dpm.REQ_ACTIVE, dpm.REQ_DONE) and st["slot"] >= 0 and st["histories"] == 20000
            with pytest.raises(RuntimeError):
                srv.submit(st["slot"], src, 1)  # a slot is not a geometry
            with pytest.raises(RuntimeError):
                srv.submit(10 ** 6, src, 1)
            while srv.status(rid)["state"] != dpm.REQ_DONE:
                srv.round()
            info = srv.info()
            assert info["n_done"] == 1 and info["n_completed"] == 1 and info["n_active"] == 0
            assert info["histories"] == srv.status(rid)["histories"] and info["gpu_ms"] > 0
            slot = srv.status(rid)["slot"]
            srv.release(rid)
            assert srv.status(rid)["state"] == dpm.REQ_RELEASED and srv.info()["n_done"] == 0
            # the released slot serves the next request of the geometry, with a clean tally
            rid2 = srv.submit(g, src, 123)
            srv.round()
            assert srv.status(rid2)["slot"] == slot
            assert srv.info()["slot_bytes"] == srv.slot_bytes(g)
        finally:
            srv.close()

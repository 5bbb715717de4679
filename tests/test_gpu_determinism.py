"""Bit-exact properties of the integer tally: the random numbers are keyed by
(seed, history, particle id) and deposits are summed in 64-bit fixed point,
so the tally cannot depend on scheduling, launch shape or kernel design."""
import numpy as np
import pytest

from paper_0910_0329_gb300 import dpm
from paper_0910_0329_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def raw_tally(wl, n, first=0, kernel=dpm.KERNEL_HISTORY, parts=None, **opts):
    with dpm.Dpm(0, W.MATERIALS, wl.params) as d:
        pid = d.load_phantom(wl.phantom)
        for f, m in (parts or [(first, n)]):
            d.run(pid, wl.source, m, wl.seed, first=f, kernel=kernel, **opts)
        _, _, raw, st = d.read(pid)
    assert st["error_flags"] == 0
    return raw


@pytest.fixture(scope="module")
def wl():
    w = W.c1_photon_wbw()
    return w


@pytest.mark.parametrize("kernel", [dpm.KERNEL_HISTORY, dpm.KERNEL_QUEUE], ids=["history", "queue"])
def test_same_seed_twice_is_bit_identical(wl, kernel):
    a = raw_tally(wl, 300000, kernel=kernel)
    b = raw_tally(wl, 300000, kernel=kernel)
    assert np.array_equal(a, b)
    c = raw_tally(W.c0_electron_wlw(), 5000, kernel=kernel)
    d = raw_tally(W.c0_electron_wlw(), 5000, kernel=kernel)
    assert np.array_equal(c, d)


@pytest.mark.parametrize("kernel", [dpm.KERNEL_HISTORY, dpm.KERNEL_QUEUE], ids=["history", "queue"])
def test_split_history_range_sums_to_the_same_tally(wl, kernel):
    a = raw_tally(wl, 200000, kernel=kernel)
    b = raw_tally(wl, 200000, kernel=kernel, parts=[(0, 70001), (70001, 129999)])
    assert np.array_equal(a, b)


def test_different_seed_differs(wl):
    a = raw_tally(wl, 20000)
    wl2 = W.c1_photon_wbw(seed=3)
    b = raw_tally(wl2, 20000)
    assert not np.array_equal(a, b)


def test_queue_kernel_equals_history_kernel(wl):
    """Same physics code, same random streams: the persistent queue kernel must
    reproduce the one-history-per-thread tally exactly."""
    a = raw_tally(wl, 300000, kernel=dpm.KERNEL_HISTORY)
    b = raw_tally(wl, 300000, kernel=dpm.KERNEL_QUEUE)
    assert np.array_equal(a, b)
    e = W.c0_electron_wlw()
    assert np.array_equal(raw_tally(e, 4000, kernel=dpm.KERNEL_HISTORY), raw_tally(e, 4000, kernel=dpm.KERNEL_QUEUE))


@pytest.mark.parametrize("shape", [dict(block_size=64, blocks_per_sm=2), dict(block_size=256, blocks_per_sm=1),
                                   dict(refill_min=1), dict(refill_min=32)])
def test_queue_launch_shape_does_not_change_the_tally(wl, shape):
    a = raw_tally(wl, 200000, kernel=dpm.KERNEL_QUEUE)
    b = raw_tally(wl, 200000, kernel=dpm.KERNEL_QUEUE, **shape)
    assert np.array_equal(a, b)


def run_stats(wl, n, kernel, **opts):
    with dpm.Dpm(0, W.MATERIALS, wl.params) as d:
        pid = d.load_phantom(wl.phantom)
        d.run(pid, wl.source, n, wl.seed, kernel=kernel, **opts)
        _, _, raw, st = d.read(pid)
    assert st["error_flags"] == 0
    return raw, st


@pytest.mark.parametrize("beam,queue_log2", [("photon", 9), ("photon", 10), ("photon", 12),
                                              ("electron", 9)])
def test_grid_phase_switches_do_not_change_the_tally(beam, queue_log2):
    """The queue kernel alternates grid-wide between a source phase and a
    secondary phase at thresholds proportional to the queue capacity; small
    queues force many switches.  The tally must still equal the per-history
    kernel's bit for bit."""
    wl = W.c1_photon_wbw() if beam == "photon" else W.c0_electron_wlw()
    n = 2_000_000 if beam == "photon" else 100_000
    ref, st_h = run_stats(wl, n, dpm.KERNEL_HISTORY)
    got, st_q = run_stats(wl, n, dpm.KERNEL_QUEUE, queue_log2=queue_log2)
    assert st_h["n_phase_switches"] == 0
    if beam == "photon":
        # 2e6 photons queue far more electrons than the threshold of these
        # capacities; an electron beam's photon backlog depends on timing
        assert st_q["n_phase_switches"] >= 2
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("config", ["6mv", "blob128"])
def test_full_size_launch_equals_history_kernel(config):
    """The benchmarked configurations at full size (10^7 histories in one
    launch with the default queue: 6 MV on the slab phantom, 20 MeV electrons
    on the 128^3 blob phantom): phase switches happen, and the tally equals
    the one-history-per-thread kernel's bit for bit."""
    wl = W.c1_photon_wbw() if config == "6mv" else W.c2_electron_blob128()
    ref, _ = run_stats(wl, wl.n_histories, dpm.KERNEL_HISTORY)
    got, st = run_stats(wl, wl.n_histories, dpm.KERNEL_QUEUE)
    assert st["n_phase_switches"] >= 2
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("order", ["denser_to_lighter", "lighter_to_denser"])
def test_update_phantom_equals_a_fresh_load(order):
    """New contents for a loaded phantom of the same size (water/bone/water
    <-> water/lung/water): the photon majorant and the tally are rebuilt, and
    the run equals one on a freshly loaded phantom bit for bit (a stale
    majorant would change the Woodcock flights; one too small would be
    wrong)."""
    a, b = W.c1_photon_wbw(), W.c0_electron_wlw()
    first, second = (a.phantom, b.phantom) if order == "denser_to_lighter" else (b.phantom, a.phantom)
    with dpm.Dpm(0, W.MATERIALS, a.params) as d:
        pid = d.load_phantom(first)
        d.run(pid, a.source, 50000, 3)
        d.update_phantom(pid, second)
        d.run(pid, a.source, 200000, 3)
        _, _, got, st = d.read(pid)
        fresh = d.load_phantom(second)
        d.run(fresh, a.source, 200000, 3)
        _, _, ref, _ = d.read(fresh)
    assert st["n_histories"] == 200000 and st["error_flags"] == 0
    assert np.array_equal(got, ref)


def test_clone_phantom_equals_a_fresh_load():
    """A device copy of a phantom (contents and majorant, empty tally) runs
    bit for bit like a freshly loaded one, also while the source phantom
    keeps its own tally."""
    wl = W.c1_photon_wbw()
    with dpm.Dpm(0, W.MATERIALS, wl.params) as d:
        src = d.load_phantom(wl.phantom)
        d.run(src, wl.source, 100000, 9)
        twin = d.clone_phantom(src)
        d.run(twin, wl.source, 200000, 3)
        _, _, got, st = d.read(twin)
        _, _, src_raw, src_st = d.read(src)
        fresh = d.load_phantom(wl.phantom)
        d.run(fresh, wl.source, 200000, 3)
        _, _, ref, _ = d.read(fresh)
    assert st["n_histories"] == 200000 and src_st["n_histories"] == 100000
    assert np.array_equal(got, ref)
    assert not np.array_equal(src_raw, ref)


@pytest.mark.parametrize("make,n", [(W.c1_photon_wbw, 200_000), (W.c0_electron_wlw, 4000)], ids=["6mv", "e20"])
def test_event_counting_changes_nothing_but_the_counts(make, n):
    """The queue kernel with and without event counts gives the same tally and
    energy counters; its counts equal the per-history kernel's (the same
    particles take the same steps), and without counting they read zero."""
    wl = make()

    def run(kernel, count):
        with dpm.Dpm(0, W.MATERIALS, wl.params) as d:
            pid = d.load_phantom(wl.phantom)
            d.run(pid, wl.source, n, wl.seed, kernel=kernel, count_events=count)
            _, _, raw, st = d.read(pid)
        assert st["error_flags"] == 0
        return raw, st

    raw0, st0 = run(dpm.KERNEL_QUEUE, 0)
    raw1, st1 = run(dpm.KERNEL_QUEUE, 1)
    rawh, sth = run(dpm.KERNEL_HISTORY, 0)
    assert np.array_equal(raw0, raw1) and np.array_equal(raw0, rawh)
    for k in ("emitted", "escaped", "missed", "deposited", "n_histories"):
        assert st0[k] == st1[k] == sth[k], k
    for k in ("n_e_steps", "n_g_flights", "n_g_interactions", "n_pushed"):
        assert st1[k] == sth[k] > 0 and st0[k] == 0, k
    assert st1["n_tally_atomics"] > 0 and st0["n_tally_atomics"] == 0


@pytest.mark.parametrize("make,n", [(W.c1_photon_wbw, 300_000), (W.c0_electron_wlw, 60_000)], ids=["6mv", "e20"])
def test_refill_pause_changes_nothing_but_the_schedule(make, n):
    """The queue kernel with the refill pause, without it and with the
    automatic choice gives the same tally and energy counters, with and
    without event counts (the pause only changes when warps look for work)."""
    wl = make()

    def run(pause, count):
        with dpm.Dpm(0, W.MATERIALS, wl.params) as d:
            pid = d.load_phantom(wl.phantom)
            d.run(pid, wl.source, n, wl.seed, refill_pause=pause, count_events=count)
            _, _, raw, st = d.read(pid)
        assert st["error_flags"] == 0
        return raw, st

    ref, st_ref = run(-1, 0)
    for pause, count in ((1, 0), (0, 0), (1, 1), (-1, 1)):
        raw, st = run(pause, count)
        assert np.array_equal(raw, ref), (pause, count)
        for k in ("emitted", "escaped", "missed", "deposited", "n_histories"):
            assert st[k] == st_ref[k], (k, pause, count)

"""Error paths of the C ABI on the GPU: argument checks, call order, and the
device-side bounded failures (queue overflow, wait time-out), which must
return an error status and leave the context usable.  No test faults, traps
or hangs the GPU: overflow and time-out are produced by tiny capacities and
wait limits that the kernel checks itself."""
import numpy as np
import pytest

from paper_0910_0329_gb300 import dpm
from paper_0910_0329_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def code_of(fn, *a, **k):
    with pytest.raises(dpm.DpmError) as e:
        fn(*a, **k)
    return e.value.code


def test_argument_and_order_errors(gpu_lib):
    wl = W.c1_photon_wbw()
    ctx = dpm.dpm_create(0)
    try:
        pid = dpm.dpm_load_phantom(ctx, wl.phantom)
        assert code_of(dpm.dpm_run, ctx, pid, wl.source, 0, 10, 1) == dpm.DPM_ESTATE  # no tables yet
        dpm.dpm_build_tables(ctx, W.MATERIALS, wl.params)
        assert code_of(dpm.dpm_run, ctx, 99, wl.source, 0, 10, 1) == dpm.DPM_EINVAL
        bad = W.Source(W.ELECTRON, W.SPEC_MONO, 50.0, wl.source.iso)
        assert code_of(dpm.dpm_run, ctx, pid, bad, 0, 10, 1) == dpm.DPM_EINVAL  # above e_max
        assert code_of(dpm.dpm_run, ctx, pid, wl.source, 0, 10, 1, dpm.run_opts(n_batches=2000)) == dpm.DPM_EINVAL
        assert code_of(dpm.dpm_run, ctx, pid, wl.source, 0, 10, 1, dpm.run_opts(physics_flags=8)) == dpm.DPM_EINVAL
        assert code_of(dpm.dpm_run, ctx, pid, wl.source, 0, 10, 1, dpm.run_opts(queue_log2=3)) == dpm.DPM_EINVAL
        ph = W.slab_phantom(2, 2, 2, 1.0, [(0, 1e9, 5, 1.0)])  # material 5 is beyond the 3 tables
        pid2 = dpm.dpm_load_phantom(ctx, ph)
        assert code_of(dpm.dpm_run, ctx, pid2, wl.source, 0, 10, 1) == dpm.DPM_EINVAL
        bad_ph = W.slab_phantom(2, 2, 2, 1.0, [(0, 1e9, 0, 1.0)])
        bad_ph.rho[3] = 0.0
        assert code_of(dpm.dpm_load_phantom, ctx, bad_ph) == dpm.DPM_EINVAL
        bad_ph.rho[3] = 1.0
        bad_ph.nx = 3000
        with pytest.raises((dpm.DpmError, ValueError)):
            dpm.dpm_load_phantom(ctx, bad_ph)
        p = dict(wl.params, n_e=10)
        assert code_of(dpm.dpm_build_tables, ctx, W.MATERIALS, p) == dpm.DPM_EINVAL
    finally:
        dpm.dpm_destroy(ctx)


def _ref_tally(wl, n):
    with dpm.Dpm(0, W.MATERIALS, wl.params) as d:
        pid = d.load_phantom(wl.phantom)
        d.run(pid, wl.source, n, wl.seed, kernel=dpm.KERNEL_HISTORY)
        return d.read(pid)[2]


def test_queue_overflow_is_reported_and_recoverable():
    wl = W.c1_photon_wbw()
    with dpm.Dpm(0, W.MATERIALS, wl.params) as d:
        pid = d.load_phantom(wl.phantom)
        d.run(pid, wl.source, 400000, wl.seed, kernel=dpm.KERNEL_QUEUE, queue_limit=1)
        with pytest.raises(dpm.DpmError) as e:
            d.read(pid)
        assert e.value.code == dpm.DPM_EQUEUE_OVERFLOW
        d.reset(pid)
        d.run(pid, wl.source, 200000, wl.seed, kernel=dpm.KERNEL_QUEUE)
        raw = d.read(pid)[2]
    assert np.array_equal(raw, _ref_tally(wl, 200000))


def test_wait_timeout_is_reported_and_recoverable():
    wl = W.c0_electron_wlw()
    with dpm.Dpm(0, W.MATERIALS, wl.params) as d:
        pid = d.load_phantom(wl.phantom)
        d.run(pid, wl.source, 20000, wl.seed, kernel=dpm.KERNEL_QUEUE, timeout_s=1e-7)
        with pytest.raises(dpm.DpmError) as e:
            d.read(pid)
        assert e.value.code == dpm.DPM_ETIMEOUT
        d.reset(pid)
        d.run(pid, wl.source, 5000, wl.seed, kernel=dpm.KERNEL_QUEUE)
        raw = d.read(pid)[2]
    assert np.array_equal(raw, _ref_tally(wl, 5000))


def test_timing_events_stay_bounded_without_reads():
    """Runs that are never read keep at most a bounded number of timing
    events; the statistics of the next read still cover every run."""
    wl = W.c1_photon_wbw()
    with dpm.Dpm(0, W.MATERIALS, wl.params) as d:
        pid = d.load_phantom(wl.phantom)
        for i in range(1100):
            d.run(pid, wl.source, 20, wl.seed, first=20 * i)
        _, _, raw, st = d.read(pid)
        assert st["n_histories"] == 22000 and st["n_transport_launches"] == 1100
        assert st["transport_ms"] > 0 and st["error_flags"] == 0
        jobs = [(pid, wl.source, 0, 20, 1)]
        for i in range(1100):
            dpm.dpm_run_batch(d.ctx, jobs, dpm.run_opts())
        bst = dpm.dpm_batch_stats(d.ctx)
        assert bst["n_transport_launches"] == 1100 and bst["transport_ms"] > 0
        assert bst["n_histories"] == 22000


def test_energy_counters_do_not_wrap_on_large_runs():
    """The run's energy counters sum the energy of every history: 2e8
    histories of 20 MeV (4e9 MeV, a beam that misses the phantom) would wrap
    an int64 counter of 2^-32 MeV quanta; the counters use 2^-24 MeV."""
    import dataclasses

    wl = W.c0_electron_wlw()
    src = dataclasses.replace(wl.source, iso=(-80.0, -80.0, 0.0))
    params = dict(wl.params, e_max=21.0)
    with dpm.Dpm(0, W.MATERIALS, params) as d:
        pid = d.load_phantom(wl.phantom)
        d.run(pid, src, 200_000_000, 3, count_events=1)
        _, _, raw, st = d.read(pid)
    assert raw.sum() == 0 and st["error_flags"] == 0
    assert st["emitted"] == pytest.approx(4.0e9, rel=1e-6)
    assert st["missed"] == st["emitted"]


def test_device_memory_budget_of_a_context(gpu_lib):
    """dpm_create's budget: allocations are counted (and released by frees),
    one that would pass the budget fails with DPM_ENOMEM before cudaMalloc,
    and the context stays usable."""
    wl = W.c0_electron_wlw()
    with dpm.Dpm(0, W.MATERIALS, wl.params) as d:
        used0, budget0 = dpm.dpm_device_bytes(d.ctx)
        assert budget0 == 0 and used0 > 0  # the tables
        pid = d.load_phantom(wl.phantom)
        used1, _ = dpm.dpm_device_bytes(d.ctx)
        V = wl.phantom.n_vox
        assert used1 - used0 >= V * (1 + 4 + 8 + 8)  # mat, rho, S1, Q
        d.run(pid, wl.source, 2000, wl.seed)
        d.read(pid)
        used_run, _ = dpm.dpm_device_bytes(d.ctx)
        need = used_run  # tables + phantom + slabs + queues of one run
        dpm.dpm_free_phantom(d.ctx, pid)
        used2, _ = dpm.dpm_device_bytes(d.ctx)
        assert used2 < used_run - V * (1 + 4 + 8 + 8)
    # a budget below what one run needs: the run fails with DPM_ENOMEM, a
    # second phantom load too, and the first phantom's tally is intact
    with dpm.Dpm(0, W.MATERIALS, wl.params, hbm_budget_bytes=need // 2) as d:
        assert dpm.dpm_device_bytes(d.ctx)[1] == need // 2
        try:
            pid = d.load_phantom(wl.phantom)
        except dpm.DpmError as e:
            assert e.code == dpm.DPM_ENOMEM
        else:
            assert code_of(d.run, pid, wl.source, 2000, wl.seed) == dpm.DPM_ENOMEM
        assert dpm.dpm_device_bytes(d.ctx)[0] <= need // 2
    # a budget that fits: the same run goes through
    with dpm.Dpm(0, W.MATERIALS, wl.params, hbm_budget_bytes=need + (1 << 20)) as d:
        pid = d.load_phantom(wl.phantom)
        d.run(pid, wl.source, 2000, wl.seed)
        assert d.read(pid)[2].sum() > 0


def test_sauter_option_is_single_run_only(gpu_lib):
    wl = W.c1_photon_wbw()
    with dpm.Dpm(0, W.MATERIALS, wl.params) as d:
        pid = d.load_phantom(wl.phantom)
        assert code_of(dpm.dpm_run_batch, d.ctx, [(pid, wl.source, 0, 100, 1)],
                       dpm.run_opts(physics_flags=dpm.SAUTER)) == dpm.DPM_EINVAL
        d.run(pid, wl.source, 1000, 1, physics_flags=dpm.SAUTER)  # a single run takes it
        assert d.read(pid)[2].sum() > 0

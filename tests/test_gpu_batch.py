"""Batched launches (dpm_run_batch): several (phantom, beam, history range)
jobs in one persistent queue launch.  Random numbers are keyed by (seed,
history, particle), so every job must reproduce, bit for bit, the integer
tally of the same job run alone with dpm_run -- with and without CUDA-graph
replay."""
import numpy as np
import pytest

from paper_0910_0329_gb300 import dpm
from paper_0910_0329_gb300 import workloads as W

pytestmark = pytest.mark.gpu
PARAMS = dict(W.DEFAULT_PARAMS, e_max=21.0)


def jobs_spec():
    c0, c1 = W.c0_electron_wlw(), W.c1_photon_wbw()
    blob = W.blob_phantom(48, 40, 56, 0.4, 17, name="blob_small")
    pencil = W.slab_phantom(21, 21, 40, 0.5, [(0, 1e9, W.MAT_WATER, 1.0)])
    X, Y, _ = pencil.extent
    return [
        (c0.phantom, c0.source, 1000, 6000, 11),
        (c1.phantom, c1.source, 0, 150000, 12),
        (blob, W.axial_source(blob, W.ELECTRON, W.SPEC_MONO, 12.0, 90.0, 100.0, 8.0, 8.0), 500, 20000, 13),
        (pencil, W.Source(W.PHOTON, W.SPEC_MONO, 15.0, (X / 2, Y / 2, 0.0), 100.0, 0.2, 0.2), 0, 60000, 14),
    ]


def alone(ph, src, first, n, seed):
    with dpm.Dpm(0, W.MATERIALS, PARAMS) as d:
        pid = d.load_phantom(ph)
        d.run(pid, src, n, seed, first=first, kernel=dpm.KERNEL_QUEUE)
        return d.read(pid)[2]


@pytest.fixture(scope="module")
def reference():
    return [alone(*j) for j in jobs_spec()]


@pytest.mark.parametrize("use_graph", [0, 1])
def test_batch_equals_jobs_run_alone(reference, use_graph):
    spec = jobs_spec()
    with dpm.Dpm(0, W.MATERIALS, PARAMS) as d:
        pids = [d.load_phantom(j[0]) for j in spec]
        jobs = [(pid, src, first, n, seed) for pid, (_, src, first, n, seed) in zip(pids, spec)]
        dpm.dpm_run_batch(d.ctx, jobs, dpm.run_opts(use_graph=use_graph, count_events=1))
        st = dpm.dpm_batch_stats(d.ctx)
        raws = [d.read(pid)[2] for pid in pids]
    assert st["error_flags"] == 0 and st["n_histories"] == sum(j[3] for j in spec)
    for got, ref in zip(raws, reference):
        assert got.sum() > 0
        assert np.array_equal(got, ref)
    dep = sum(r.sum() for r in raws) / 2.0 ** 32
    assert abs(st["emitted"] - dep - st["escaped"] - st["missed"]) / st["emitted"] < 1e-5


def test_graph_replay_with_new_ranges_and_recapture():
    spec = jobs_spec()[:2]
    with dpm.Dpm(0, W.MATERIALS, PARAMS) as d:
        pids = [d.load_phantom(j[0]) for j in spec]
        for rep in range(3):  # replays with new history ranges and seeds kept
            jobs = [(pid, src, first + rep * n, n, seed) for pid, (_, src, first, n, seed) in zip(pids, spec)]
            dpm.dpm_run_batch(d.ctx, jobs, dpm.run_opts(use_graph=1))
        # a different shape (history count) forces a new capture
        jobs = [(pid, src, first + 3 * n, n // 2, seed) for pid, (_, src, first, n, seed) in zip(pids, spec)]
        dpm.dpm_run_batch(d.ctx, jobs, dpm.run_opts(use_graph=1))
        st = dpm.dpm_batch_stats(d.ctx)
        raws = [d.read(pid)[2] for pid in pids]
    assert st["error_flags"] == 0
    for (ph, src, first, n, seed), got in zip(spec, raws):
        with dpm.Dpm(0, W.MATERIALS, PARAMS) as d:
            pid = d.load_phantom(ph)
            d.run(pid, src, 3 * n, seed, first=first)
            d.run(pid, src, n // 2, seed, first=first + 3 * n)
            ref = d.read(pid)[2]
        assert np.array_equal(got, ref)


def test_batch_argument_errors():
    spec = jobs_spec()
    with dpm.Dpm(0, W.MATERIALS, PARAMS) as d:
        pid = d.load_phantom(spec[0][0])
        with pytest.raises(dpm.DpmError) as e:
            dpm.dpm_run_batch(d.ctx, [(pid, spec[0][1], 0, 10, 1), (pid, spec[0][1], 10, 10, 1)])
        assert e.value.code == dpm.DPM_EINVAL
        with pytest.raises(dpm.DpmError) as e:
            dpm.dpm_run_batch(d.ctx, [(pid, spec[0][1], 0, 10, 1)], dpm.run_opts(kernel=dpm.KERNEL_HISTORY))
        assert e.value.code == dpm.DPM_EINVAL
        with pytest.raises(dpm.DpmError) as e:
            dpm.dpm_run_batch(d.ctx, [(pid + 7, spec[0][1], 0, 10, 1)])
        assert e.value.code == dpm.DPM_EINVAL
        dpm.dpm_run_batch(d.ctx, [])  # empty batch is a no-op
        dpm.dpm_run_batch(d.ctx, [(pid, spec[0][1], 0, 0, 1)])  # so is a job without histories


def test_large_batch_with_phase_switches_equals_jobs_run_alone():
    """Enough histories per job, and a small enough queue, for the grid-wide
    phase to switch within the shared launch, across photon-beam and
    electron-beam jobs (jobs below 10^6 histories share the launch)."""
    c1, c0 = W.c1_photon_wbw(), W.c0_electron_wlw()
    blob = W.blob_phantom(64, 64, 64, 0.4, 23, name="blob64")
    spec = [(c1.phantom, c1.source, 0, 900_000, 21),
            (blob, W.axial_source(blob, W.PHOTON, W.SPEC_6MV, 6.0, 90.0, 100.0, 10.0, 10.0), 0, 900_000, 22),
            (c0.phantom, c0.source, 0, 200_000, 23)]
    ref = [alone(*j) for j in spec]
    with dpm.Dpm(0, W.MATERIALS, PARAMS) as d:
        pids = [d.load_phantom(j[0]) for j in spec]
        jobs = [(pid, src, first, n, seed) for pid, (_, src, first, n, seed) in zip(pids, spec)]
        dpm.dpm_run_batch(d.ctx, jobs, dpm.run_opts(queue_log2=11))
        st = dpm.dpm_batch_stats(d.ctx)
        raws = [d.read(pid)[2] for pid in pids]
    assert st["error_flags"] == 0 and st["n_phase_switches"] >= 2
    for got, r in zip(raws, ref):
        assert np.array_equal(got, r)


def test_autotuned_batch_keeps_the_tally(tmp_path):
    """The autotuner times trial batches through the C ABI, resets the
    tallies it touched and returns options from its search space; the batch
    run with them reproduces the default launch's tally bit for bit."""
    from paper_0910_0329_gb300 import autotune

    spec = jobs_spec()[:3]
    space = {"queue_log2": [12, 14], "blocks_per_sm": [6, 8], "refill_min": [8]}
    with dpm.Dpm(0, W.MATERIALS, PARAMS) as d:
        pids = [d.load_phantom(j[0]) for j in spec]
        jobs = [(pid, src, first, n, seed) for pid, (_, src, first, n, seed) in zip(pids, spec)]
        opts = autotune.tune_batch(d, jobs, "test-gpu", "three-jobs", fraction=0.5, space=space,
                                   cache_path=str(tmp_path / "tune.json"))
        assert all(opts[k] in v for k, v in space.items())
        assert all(d.read(pid)[2].sum() == 0 for pid in pids)  # trial tallies were reset
        assert autotune.load(autotune.signature("test-gpu", "three-jobs"), str(tmp_path / "tune.json"))["opts"] == opts
        dpm.dpm_run_batch(d.ctx, jobs, dpm.run_opts(**opts))
        dpm.dpm_batch_stats(d.ctx)
        tuned = [d.read(pid)[2] for pid in pids]
        for pid in pids:
            dpm.dpm_reset_tally(d.ctx, pid)
        dpm.dpm_run_batch(d.ctx, jobs, dpm.run_opts())
        dpm.dpm_batch_stats(d.ctx)
        plain = [d.read(pid)[2] for pid in pids]
    for a, b in zip(tuned, plain):
        assert np.array_equal(a, b)


def test_large_jobs_get_their_own_launch_and_keep_the_tally():
    """A job of 10^6 histories or more runs as a launch of its own inside the
    batch (and its graph); its tally still equals the job run alone."""
    c1 = W.c1_photon_wbw()
    blob = W.blob_phantom(48, 48, 48, 0.4, 31, name="blob48")
    spec = [(c1.phantom, c1.source, 500, 1_200_000, 41),
            (blob, W.axial_source(blob, W.ELECTRON, W.SPEC_MONO, 9.0, 90.0, 100.0, 8.0, 8.0), 0, 30_000, 42)]
    ref = [alone(*j) for j in spec]
    for use_graph in (0, 1):
        with dpm.Dpm(0, W.MATERIALS, PARAMS) as d:
            pids = [d.load_phantom(j[0]) for j in spec]
            jobs = [(pid, src, first, n, seed) for pid, (_, src, first, n, seed) in zip(pids, spec)]
            dpm.dpm_run_batch(d.ctx, jobs, dpm.run_opts(use_graph=use_graph))
            st = dpm.dpm_batch_stats(d.ctx)
            raws = [d.read(pid)[2] for pid in pids]
        assert st["error_flags"] == 0 and st["n_histories"] == 1_230_000
        for got, r in zip(raws, ref):
            assert np.array_equal(got, r)

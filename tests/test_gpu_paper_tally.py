"""The paper's own tally (Sec. 2.4) as an ablation of the exact one: one
history per thread, a sparse per-thread (voxel, energy) counter emptied into
float slabs with atomic float additions (native, or a compare-and-swap loop).
The device physics and random numbers are those of the other kernels, so the
trajectories are the same: the event and energy counters must match the
one-history-per-thread kernel exactly, and each voxel's energy must equal its
exact fixed-point sum up to the rounding of the float additions."""
import numpy as np
import pytest

from paper_0910_0329_gb300 import dpm
from paper_0910_0329_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U = 2.0 ** -24  # unit roundoff of float
SAME = ["emitted", "escaped", "missed", "n_e_steps", "n_g_flights", "n_g_interactions", "n_pushed", "n_histories"]


def tallies(wl, n, kernel):
    with dpm.Dpm(0, W.MATERIALS, wl.params) as d:
        pid = d.load_phantom(wl.phantom)
        d.run(pid, wl.source, n, wl.seed, kernel=dpm.KERNEL_HISTORY, n_batches=1)
        _, _, exact, st_exact = d.read(pid)
        d.reset(pid)
        d.run(pid, wl.source, n, wl.seed, kernel=kernel, n_batches=1)
        _, _, flt, st_flt = d.read(pid)
    return exact.astype(np.float64), st_exact, flt.astype(np.float64), st_flt


@pytest.mark.parametrize("kernel", [dpm.KERNEL_PAPER_F32, dpm.KERNEL_PAPER_CAS], ids=["f32", "cas"])
@pytest.mark.parametrize("case,n", [("6mv", 200_000), ("e20", 20_000)])
def test_float_tally_equals_the_exact_one_up_to_float_rounding(kernel, case, n):
    wl = W.c1_photon_wbw() if case == "6mv" else W.c0_electron_wlw()
    exact, st_e, flt, st_f = tallies(wl, n, kernel)
    for k in SAME:
        assert st_f[k] == st_e[k], k
    assert st_f["error_flags"] == 0 and st_e["error_flags"] == 0
    # the float counter empties at least one entry per history that deposits
    assert st_f["n_tally_atomics"] > 0
    # per voxel: a chain of at most n + m float additions of positive terms
    # (one per history into the slab, m within one history's counter entry)
    # errs by at most gamma_(n+m) of the sum.  m is below the steps of one
    # history, whose mean is checked to stay far below 4096.  The final
    # rounding to 2^-32 MeV and the exact tally's per-deposit rounding (half a
    # unit each) are covered by an absolute 2^20 units (2^-12 MeV).
    steps = (st_e["n_e_steps"] + st_e["n_g_flights"]) / n
    assert steps < 4096
    k = n + 4096
    gamma = k * U / (1 - k * U)
    assert np.all(np.abs(flt - exact) <= gamma * exact + 2.0 ** 20), np.max(np.abs(flt - exact) / np.maximum(exact, 1))
    # what rounding errors actually do: far below the bound
    hot = exact > 0.1 * exact.max()
    rel = np.abs(flt[hot] - exact[hot]) / exact[hot]
    assert np.median(rel) < 1e-4
    assert abs(flt.sum() - exact.sum()) <= 1e-4 * exact.sum()


def test_float_tally_is_rejected_outside_dpm_run():
    wl = W.c0_electron_wlw()
    with dpm.Dpm(0, W.MATERIALS, wl.params) as d:
        pid = d.load_phantom(wl.phantom)
        with pytest.raises(dpm.DpmError):
            dpm.dpm_run_batch(d.ctx, [(pid, wl.source, 0, 100, 1)], dpm.run_opts(kernel=dpm.KERNEL_PAPER_F32))
        with pytest.raises(dpm.DpmError):
            d.run(pid, wl.source, 100, 1, kernel=7)

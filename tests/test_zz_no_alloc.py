"""The transport entry point that allocates no device memory.

It exists for callers that cannot call cudaMalloc while they run: programs
whose device memory belongs to a pool or arena that refuses further device
allocations, or that work inside a fixed device-memory budget.  It must give
the same integer tally as dpm_run() (same physics, same random numbers), here
checked exactly on two calls in a row into the same caller-owned buffer, and
the device's free memory must not move across either call (the fixed scratch
and the kernels were loaded by dpm_create).  This file is collected last so
that a run stopping at the first failure has already run every other test."""
import math

import numpy as np
import pytest

from paper_0910_0329_gb300 import dpm
from paper_0910_0329_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _free_bytes(torch):
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info(0)[0]


@pytest.mark.parametrize("make,n", [(W.c1_photon_wbw, 200_000), (W.c0_electron_wlw, 5_000)])
def test_noalloc_matches_dpm_run_on_two_calls(gpu_lib, make, n):
    import torch

    wl = make()
    ph = wl.phantom
    with dpm.Dpm(0, W.MATERIALS, wl.params) as d:
        pid = d.load_phantom(ph)
        tally = torch.zeros(ph.n_vox, dtype=torch.int64, device="cuda:0")
        # first call: histories [0, n); no device memory taken
        f0 = _free_bytes(torch)
        st1 = dpm.dpm_run_noalloc(d.ctx, pid, wl.source, 0, n, wl.seed, tally.data_ptr())
        assert _free_bytes(torch) == f0
        got1 = tally.cpu().numpy().copy()
        d.run(pid, wl.source, n, wl.seed, first=0, kernel=dpm.KERNEL_QUEUE, count_events=1)
        ref1 = d.read(pid)
        assert got1.sum() > 0
        assert np.array_equal(got1, ref1[2])
        # the counters match the same run through dpm_run; deposited is the tally's
        st_ref = ref1[3]
        assert st1["error_flags"] == 0 and math.isnan(st1["deposited"])
        for k in ("emitted", "escaped", "missed"):
            assert st1[k] == st_ref[k]
        for k in ("n_e_steps", "n_g_flights", "n_g_interactions", "n_tally_atomics", "n_pushed"):
            assert st1[k] == st_ref[k]
        dep = got1.sum(dtype=np.float64) / 2.0 ** 32
        assert abs(st1["emitted"] - dep - st1["escaped"] - st1["missed"]) < 1e-5 * st1["emitted"]
        # second call in a row: histories [n, 2n), added to the same buffer
        f1 = _free_bytes(torch)
        dpm.dpm_run_noalloc(d.ctx, pid, wl.source, n, n, wl.seed, tally.data_ptr())
        assert _free_bytes(torch) == f1
        got2 = tally.cpu().numpy()
        d.run(pid, wl.source, n, wl.seed, first=n, kernel=dpm.KERNEL_QUEUE)
        ref2 = d.read(pid)[2]  # the context's tally now holds [0, 2n)
        assert np.array_equal(got2, ref2)

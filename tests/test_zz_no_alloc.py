"""The transport entry point that allocates no device memory.

It exists for callers that cannot call cudaMalloc while they run: programs
whose device memory belongs to a pool or arena that refuses further device
allocations, or that work inside a fixed device-memory budget.  It must give
the same integer tally as dpm_run() (same physics, same random numbers), here
checked exactly on two calls in a row into the same caller-owned buffer.
This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

from paper_0910_0329_gb300 import dpm
from paper_0910_0329_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("make,n", [(W.c1_photon_wbw, 200_000), (W.c0_electron_wlw, 5_000)])
def test_noalloc_matches_dpm_run_on_two_calls(gpu_lib, make, n):
    import torch

    wl = make()
    ph = wl.phantom
    with dpm.Dpm(0, W.MATERIALS, wl.params) as d:
        pid = d.load_phantom(ph)
        tally = torch.zeros(ph.n_vox, dtype=torch.int64, device="cuda:0")
        torch.cuda.synchronize()
        # first call: histories [0, n)
        dpm.dpm_run_noalloc(d.ctx, pid, wl.source, 0, n, wl.seed, tally.data_ptr())
        got1 = tally.cpu().numpy().copy()
        d.run(pid, wl.source, n, wl.seed, first=0, kernel=dpm.KERNEL_QUEUE)
        ref1 = d.read(pid)[2]
        assert got1.sum() > 0
        assert np.array_equal(got1, ref1)
        # second call in a row: histories [n, 2n), added to the same buffer
        dpm.dpm_run_noalloc(d.ctx, pid, wl.source, n, n, wl.seed, tally.data_ptr())
        got2 = tally.cpu().numpy()
        d.run(pid, wl.source, n, wl.seed, first=n, kernel=dpm.KERNEL_QUEUE)
        ref2 = d.read(pid)[2]  # the context's tally now holds [0, 2n)
        assert np.array_equal(got2, ref2)

"""The cost of single precision (Sec. 2.3 transports in FP32): the
per-history kernel instantiated in FP64, with FP64 tables, against the FP32
kernel on the same seeds and history ranges, per configuration.  The two
draw the same random numbers, so their tallies are strongly correlated and
their difference measures the FP32 rounding (tables and arithmetic), not the
statistics.  Measured on GB300: the integral energy per history differs by
about 1e-6, the per-voxel difference is 0.01-0.09 of the statistical sigma,
the largest depth-dose plane difference 3e-4 of the largest plane.  Bounds:
1e-5 on the integral, a quarter sigma per voxel, 0.2 % per plane."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_0910_0329_gb300 import dpm
from paper_0910_0329_gb300 import workloads as W

from parity_util import compare

pytestmark = pytest.mark.gpu

# config -> (workload, histories)
CONFIGS = {
    "e20_wlw_61x61x60": (W.c0_electron_wlw, 400_000),
    "6mv_wbw_61x61x60": (W.c1_photon_wbw, 10_000_000),
    "e20_blob128": (W.c2_electron_blob128, 1_000_000),
}


def run(wl, n, kernel):
    with dpm.Dpm(0, W.MATERIALS, wl.params) as d:
        pid = d.load_phantom(wl.phantom)
        d.run(pid, wl.source, n, wl.seed, kernel=kernel, n_batches=50)
        return d.read(pid)


@pytest.mark.parametrize("name", list(CONFIGS))
def test_fp32_against_fp64_transport(name):
    make, n = CONFIGS[name]
    wl = make()
    d32, s32, raw32, st32 = run(wl, n, dpm.KERNEL_HISTORY)
    d64, s64, raw64, st64 = run(wl, n, dpm.KERNEL_HISTORY_F64)
    assert st32["error_flags"] == 0 and st64["error_flags"] == 0
    # the same source particles: emitted energy to FP32 rounding of the energies
    assert st64["emitted"] == pytest.approx(st32["emitted"], rel=1e-6)
    bal = abs(st64["emitted"] - st64["deposited"] - st64["escaped"] - st64["missed"]) / st64["emitted"]
    assert bal < 1e-7
    e32 = raw32.sum() / 2.0 ** 32 / n
    e64 = raw64.sum() / 2.0 ** 32 / n
    rel = (e32 - e64) / e64
    sel = d64 > 0.1 * d64.max()
    z = (d32[sel] - d64[sel]) / np.sqrt(s32[sel] ** 2 + s64[sel] ** 2)
    # depth dose (lateral planes), relative to the largest plane
    p32 = raw32.reshape(wl.phantom.nz, -1).sum(axis=1).astype(np.float64)
    p64 = raw64.reshape(wl.phantom.nz, -1).sum(axis=1).astype(np.float64)
    plane_rel = np.abs(p32 - p64).max() / p64.max()
    print(f"{name}: n={n} integral FP32-FP64 {rel:+.2e}; voxels (D>10% Dmax) {sel.sum()}: "
          f"z mean {z.mean():+.4f} std {z.std():.4f} max|z| {np.abs(z).max():.3f}; "
          f"max plane diff {plane_rel:.2e} of the largest plane; fp64 balance {bal:.1e}")
    assert abs(rel) < 1e-5
    assert abs(z.mean()) < 0.02 and z.std() < 0.25 and plane_rel < 2e-3


def test_fp64_kernel_matches_the_oracle():
    """The FP64 kernel is the FP32 code in double precision: it agrees with
    the oracle by the parity criterion of the FP32 kernels."""
    wl = W.c0_electron_wlw()
    orc = O.run(wl.phantom, W.MATERIALS, wl.params, wl.source, 80000, 1000 + wl.seed)
    n = 800_000
    dose, sigma, raw, st = run(wl, n, dpm.KERNEL_HISTORY_F64)
    r = compare(wl.phantom, dose, sigma, raw, n, orc)
    print(r)
    assert r["pass_frac"] >= 0.95 and abs(r["e_rel_diff"]) < 0.2e-2, r


def test_fp64_kernel_is_rejected_outside_dpm_run():
    wl = W.c0_electron_wlw()
    with dpm.Dpm(0, W.MATERIALS, wl.params) as d:
        pid = d.load_phantom(wl.phantom)
        with pytest.raises(dpm.DpmError):
            dpm.dpm_run_batch(d.ctx, [(pid, wl.source, 0, 100, 1)], dpm.run_opts(kernel=dpm.KERNEL_HISTORY_F64))

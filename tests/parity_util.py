"""Helpers for the statistical dose comparison between the CUDA path and the
oracle (test infrastructure)."""
import math

import numpy as np

MEV_J = 1.602176634e-13


def gy_per_mev(ph):
    return MEV_J / (ph.rho.astype(np.float64) * ph.dx * ph.dy * ph.dz * 1e-3)


def compare(ph, dose_g, sigma_g, raw_g, n_g, orc, frac_cut=0.1):
    """Voxel z-scores z = (D_gpu - D_oracle)/sqrt(s_gpu^2 + s_oracle^2) over
    voxels with D > frac_cut * Dmax, and the integral energy per history."""
    conv = gy_per_mev(ph)
    d_o = orc.S1 / orc.n * conv
    s_o = orc.sigma_mean_energy() * conv
    dmax = dose_g.max()
    sel = dose_g > frac_cut * dmax
    z = (dose_g[sel] - d_o[sel]) / np.sqrt(sigma_g[sel] ** 2 + s_o[sel] ** 2 + 1e-300)
    e_g = raw_g.sum() / 2.0 ** 32 / n_g
    e_o, se_o = orc.total_energy_and_sigma()
    # the GPU's standard error of the total, from the oracle's per-history spread
    se_g = se_o * math.sqrt(orc.n / n_g)
    return {
        "n_vox": int(sel.sum()),
        "pass_frac": float(np.mean(np.abs(z) <= 2.0)),
        "z_mean": float(z.mean()),
        "z_std": float(z.std()),
        "e_gpu": e_g,
        "e_oracle": e_o,
        "e_rel_diff": (e_g - e_o) / e_o,
        "e_rel_sigma": math.sqrt(se_o ** 2 + se_g ** 2) / e_o,
    }

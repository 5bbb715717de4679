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


def compare_planes(ph, raw_g, n_g, orc, frac_cut=0.1):
    """Depth-dose integrated over each z plane: the GPU's and the oracle's
    energy per history in every plane with more than frac_cut of the largest
    plane's, z = (E_gpu - E_oracle) / sigma with the oracle's history-by-history
    standard deviation of the plane energy scaled to both history counts (the
    same physics on both sides), and the relative differences of the planes
    whose combined 2 sigma is below 0.2 %."""
    nz = ph.nz
    e_o, se_o = orc.plane_energy_and_sigma(nz)
    sd_h = se_o * math.sqrt(max(orc.n - 1, 1))  # per-history standard deviation
    e_g = raw_g.reshape(nz, -1).sum(axis=1).astype(np.float64) / 2.0 ** 32 / n_g
    sel = e_o > frac_cut * e_o.max()
    sig = sd_h[sel] * math.sqrt(1.0 / orc.n + 1.0 / n_g)
    z = (e_g[sel] - e_o[sel]) / sig
    rel = (e_g[sel] - e_o[sel]) / e_o[sel]
    tight = 2 * sig / e_o[sel] < 0.2e-2
    return {
        "n_planes": int(sel.sum()),
        "pass_frac": float(np.mean(np.abs(z) <= 2.0)),
        "z_max": float(np.abs(z).max()),
        "z_mean": float(z.mean()),
        "chi2_per_plane": float(np.mean(z * z)),
        "z": [round(float(x), 2) for x in z],
        "rel_sigma_median": float(np.median(sig / e_o[sel])),
        "n_tight": int(tight.sum()),
        "rel_max_tight": float(np.abs(rel[tight]).max()) if tight.any() else 0.0,
    }

"""GPU parity of the random-number generator and of the device tables against
the FP64 oracle, element by element (through the C ABI diagnostics)."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_0910_0329_gb300 import dpm
from paper_0910_0329_gb300 import workloads as W

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
P = W.DEFAULT_PARAMS
M32 = 0xFFFFFFFF


def philox_ref(c, k):
    """Philox4x32-10 written from its published definition (Salmon et al. 2011)."""
    c, k = list(c), list(k)
    for r in range(10):
        if r:
            k = [(k[0] + 0x9E3779B9) & M32, (k[1] + 0xBB67AE85) & M32]
        p0, p1 = 0xD2511F53 * c[0], 0xCD9E8D57 * c[2]
        c = [((p1 >> 32) ^ c[1] ^ k[0]) & M32, p1 & M32, ((p0 >> 32) ^ c[3] ^ k[1]) & M32, p0 & M32]
    return c


def test_philox_python_reference_matches_published_vectors():
    for line in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        assert philox_ref(w[0:4], w[4:6]) == w[6:10]


def test_gpu_philox_bit_exact(tables_ctx):
    rows = [[int(x, 16) for x in l.split()] for l in open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    rng = np.random.default_rng(5)
    ctr = np.concatenate([np.array([r[0:4] for r in rows], np.uint32), rng.integers(0, 2 ** 32, (997, 4), np.uint32)])
    key = np.concatenate([np.array([r[4:6] for r in rows], np.uint32), rng.integers(0, 2 ** 32, (997, 2), np.uint32)])
    out = dpm.dpm_diag_philox(tables_ctx.ctx, ctr, key)
    for i in range(len(ctr)):
        assert list(out[i]) == philox_ref(ctr[i].tolist(), key[i].tolist())


def energies(lo, hi, n=400):
    return np.geomspace(lo, hi, n)


def mats():
    return [O.material(m) for m in W.MATERIALS]


def grid(params=P):
    """Energy nodes of the per-material tables (documented in include/dpm.h)."""
    e_lo, e_hi = 0.99 * min(params["eabs_e"], params["eabs_g"]), 1.01 * params["e_max"]
    return np.exp(np.linspace(np.log(e_lo), np.log(e_hi), int(params["n_e"])))


# The device finds a table position with the hardware logarithm: within
# 7.2e-7 of ln E on the tables' range (3 ulp of |ln E| < 4, or 2^-21.41 on
# [0.5, 2], the intrinsic's documented bounds), i.e. at most this many node
# spacings off at the default grid.
POS_ERR = 7.2e-7 * (P["n_e"] - 1) / math.log(1.01 * P["e_max"] / (0.99 * min(P["eabs_e"], P["eabs_g"])))


def interp_tolerance(f, E, params=P):
    """Bound on linear interpolation in ln E of the oracle function f at E: a
    quarter of the largest second difference of f over the two node intervals
    around E (h^2/8 f'' for smooth f, h/4 times the slope jump at a kink),
    the position error of the device's logarithm times the largest first
    difference, plus FP32 storage rounding."""
    g = grid(params)
    i = np.clip(np.searchsorted(g, E) - 1, 1, len(g) - 3)
    f0, f1, f2, f3 = (np.array([f(g[j]) for j in i + k]) for k in (-1, 0, 1, 2))
    d2 = np.maximum(np.abs(f2 - 2 * f1 + f0), np.abs(f3 - 2 * f2 + f1))
    d1 = np.maximum(np.maximum(np.abs(f1 - f0), np.abs(f2 - f1)), np.abs(f3 - f2))
    return d2 / 4.0 + POS_ERR * d1 + 4e-7 * np.maximum(np.abs(f1), np.abs(f2))


def check(got, f, E):
    ref = np.array([f(e) for e in E])
    tol = interp_tolerance(f, E)
    bad = np.abs(got - ref) > tol
    assert not bad.any(), list(zip(E[bad][:5], got[bad][:5], ref[bad][:5], tol[bad][:5]))


@pytest.mark.parametrize("m", [0, 1, 2])
def test_photon_coefficients(tables_ctx, m):
    L, mm = O.lib(), mats()[m]
    E = energies(0.051, 20.5)
    mc = lambda e: L.or_mu_compton(mm, e)
    mp = lambda e: L.or_mu_photo(mm, e, P["c_pe"])
    mt = lambda e: mc(e) + mp(e) + L.or_mu_pair(mm, e)
    ctx = tables_ctx.ctx
    check(dpm.dpm_diag_table(ctx, 0, m, E), mt, E)
    check(dpm.dpm_diag_table(ctx, 1, m, E), lambda e: mc(e) / mt(e), E)
    check(dpm.dpm_diag_table(ctx, 2, m, E), lambda e: mp(e) / mt(e), E)


@pytest.mark.parametrize("m", [0, 2])
def test_electron_tables(tables_ctx, m):
    L, mm = O.lib(), mats()[m]
    pr = O.params(P)
    E = energies(0.2, 20.5)
    ctx = tables_ctx.ctx
    e_lo = 0.99 * min(P["eabs_e"], P["eabs_g"])
    check(dpm.dpm_diag_table(ctx, 4, m, E), lambda e: L.or_scol(mm, e, P["wcc"]) + L.or_srad(mm, e, P["wcr"]), E)
    check(dpm.dpm_diag_table(ctx, 3, m, E), lambda e: L.or_csda_path(mm, pr, e_lo, e), E)
    sig = lambda e: L.or_moller_sigma(mm, e, P["wcc"]) + L.or_brems_sigma(mm, e, P["wcr"])
    check(dpm.dpm_diag_table(ctx, 5, m, E), sig, E)
    check(dpm.dpm_diag_table(ctx, 7, m, E), lambda e: L.or_moller_sigma(mm, e, P["wcc"]) / sig(e) if sig(e) > 0 else 0.0,
          E)
    check(dpm.dpm_diag_table(ctx, 6, m, E), lambda e: L.or_lambda1_inv(mm, e), E)


@pytest.mark.parametrize("m", [0, 2])
def test_csda_energy_loss(tables_ctx, m):
    """Energy after a mass path, as the electron step computes it (range
    table + Newton), against the oracle's exact CSDA solution.  Paths up to
    the 5 % energy-loss step."""
    L, mm = O.lib(), mats()[m]
    pr = O.params(P)
    E = energies(0.21, 20.0, 200)
    path = np.array([L.or_csda_path(mm, pr, 0.95 * e, e) for e in E]) * np.linspace(0.02, 1.0, len(E))
    ref = np.array([L.or_csda_energy(mm, pr, e, s) for e, s in zip(E, path)])
    got = dpm.dpm_diag_table(tables_ctx.ctx, 8, m, E, path)
    # compare the energy lost: relative error of the loss, bounded by the
    # table's range accuracy divided by the (small) relative loss
    np.testing.assert_allclose(E - got, E - ref, rtol=2e-3, atol=2e-6 * E.max())


def test_photon_majorant_dominates(tables_ctx):
    ph = W.c1_photon_wbw(10).phantom
    pid = tables_ctx.load_phantom(ph)
    E = np.geomspace(0.051, 6.4, 3000)
    mm = dpm.dpm_diag_table(tables_ctx.ctx, 9, pid, E)
    for m, rho in [(W.MAT_WATER, 1.0), (W.MAT_BONE, 1.85)]:
        mu = dpm.dpm_diag_table(tables_ctx.ctx, 0, m, E) * rho
        assert (mm >= mu * (1 - 1e-7)).all()
    dpm.dpm_free_phantom(tables_ctx.ctx, pid)

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


# energies spanning the tables, avoiding one grid interval around the kinks of
# the stopping power (T = 2 wcc, T = wcr) where linear interpolation is
# first-order
def energies(lo, hi, n=400, avoid=()):
    e = np.geomspace(lo, hi, n)
    keep = np.ones(n, bool)
    for a in avoid:
        keep &= np.abs(np.log(e / a)) > 0.01
    return e[keep]


def mats():
    return [O.material(m) for m in W.MATERIALS]


# Tolerances: linear interpolation on a ln E grid of spacing h = ln(e_hi/e_lo)/(n_e-1)
# has relative error h^2/8 * |(ln f)''| + FP32 rounding; for these smooth
# coefficients (powers up to E^-3) that is below 3e-5 at n_e = 2048.
REL = 3e-5


@pytest.mark.parametrize("m", [0, 1, 2])
def test_photon_coefficients(tables_ctx, m):
    L, mm = O.lib(), mats()[m]
    E = energies(0.051, 20.5)
    mu = np.array([L.or_mu_compton(mm, e) + L.or_mu_photo(mm, e, P["c_pe"]) + L.or_mu_pair(mm, e) for e in E])
    pc = np.array([L.or_mu_compton(mm, e) for e in E]) / mu
    ppe = np.array([L.or_mu_photo(mm, e, P["c_pe"]) for e in E]) / mu
    ctx = tables_ctx.ctx
    np.testing.assert_allclose(dpm.dpm_diag_table(ctx, 0, m, E), mu, rtol=REL)
    np.testing.assert_allclose(dpm.dpm_diag_table(ctx, 1, m, E), pc, rtol=REL, atol=2e-6)
    np.testing.assert_allclose(dpm.dpm_diag_table(ctx, 2, m, E), ppe, rtol=REL, atol=2e-6)


@pytest.mark.parametrize("m", [0, 2])
def test_electron_tables(tables_ctx, m):
    L, mm = O.lib(), mats()[m]
    pr = O.params(P)
    E = energies(0.2, 20.5, avoid=(2 * P["wcc"], P["wcr"]))
    ctx = tables_ctx.ctx
    e_lo = 0.99 * min(P["eabs_e"], P["eabs_g"])
    S = np.array([L.or_scol(mm, e, P["wcc"]) + L.or_srad(mm, e, P["wcr"]) for e in E])
    np.testing.assert_allclose(dpm.dpm_diag_table(ctx, 4, m, E), S, rtol=REL)
    R = np.array([L.or_csda_path(mm, pr, e_lo, e) for e in E])
    np.testing.assert_allclose(dpm.dpm_diag_table(ctx, 3, m, E), R, rtol=REL)
    sm = np.array([L.or_moller_sigma(mm, e, P["wcc"]) for e in E])
    sb = np.array([L.or_brems_sigma(mm, e, P["wcr"]) for e in E])
    np.testing.assert_allclose(dpm.dpm_diag_table(ctx, 5, m, E), sm + sb, rtol=REL, atol=1e-7)
    np.testing.assert_allclose(dpm.dpm_diag_table(ctx, 7, m, E), np.where(sm + sb > 0, sm / (sm + sb), 0),
                               rtol=REL, atol=2e-6)
    l1 = np.array([L.or_lambda1_inv(mm, e) for e in E])
    np.testing.assert_allclose(dpm.dpm_diag_table(ctx, 6, m, E), l1, rtol=REL)


@pytest.mark.parametrize("m", [0, 2])
def test_csda_energy_loss(tables_ctx, m):
    """Energy after a mass path, as the electron step computes it (range
    table + Newton), against the oracle's exact CSDA solution.  Paths up to
    the 5 % energy-loss step."""
    L, mm = O.lib(), mats()[m]
    pr = O.params(P)
    E = energies(0.21, 20.0, 200, avoid=(2 * P["wcc"],))
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

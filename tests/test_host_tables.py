"""CPU checks of the table builder (host logic of the CUDA library, read through
include/dpm_host.h without a GPU) against the oracle's FP64 closed forms.

The device interpolates the per-material tables linearly in ln E and the
sampling tables bilinearly in (ln E, u); this file reproduces that lookup in
numpy and bounds the error by the interpolation error of the oracle function
itself (second differences on the same grid), so a wrong term in the builder
shows up as a violation far above the bound."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_0910_0329_gb300 import build_lib, dpm
from paper_0910_0329_gb300 import workloads as W

P = W.DEFAULT_PARAMS
MC2 = 0.51099895


@pytest.fixture(scope="module")
def tabs():
    build_lib.build()
    t = dpm.HostTables(W.MATERIALS, P)
    yield t
    t.close()


def lin_lookup(tab, meta, m, col, E):
    """Per-material table value as the device computes it (el_at / ph_at)."""
    e_lo, e_hi, n = meta[0], meta[1], int(meta[2])
    a = tab.reshape(-1, n, 4)[m, :, col].astype(np.float64) if tab.size % (4 * n) == 0 and col >= 0 else \
        tab.reshape(-1, n)[m].astype(np.float64)
    x = (np.log(E) - math.log(e_lo)) * (n - 1) / (math.log(e_hi) - math.log(e_lo))
    x = np.clip(x, 0, n - 1 - 1e-3)
    i = x.astype(int)
    f = x - i
    return a[i] + f * (a[i + 1] - a[i])


def grid(meta):
    return np.exp(np.linspace(math.log(meta[0]), math.log(meta[1]), int(meta[2])))


def tol(f, E, meta):
    g = grid(meta)
    i = np.clip(np.searchsorted(g, E) - 1, 1, len(g) - 3)
    f0, f1, f2, f3 = (np.array([f(g[j]) for j in i + k]) for k in (-1, 0, 1, 2))
    d2 = np.maximum(np.abs(f2 - 2 * f1 + f0), np.abs(f3 - 2 * f2 + f1))
    return d2 / 4.0 + 4e-7 * np.maximum(np.abs(f1), np.abs(f2))


def check(got, f, E, meta):
    ref = np.array([f(e) for e in E])
    bad = np.abs(got - ref) > tol(f, E, meta)
    assert not bad.any(), list(zip(E[bad][:4], got[bad][:4], ref[bad][:4]))


def test_builder_rejects_bad_input():
    build_lib.build()
    with pytest.raises(dpm.DpmError):
        dpm.HostTables(W.MATERIALS, dict(P, n_e=10))
    with pytest.raises(dpm.DpmError):
        dpm.HostTables(W.MATERIALS, dict(P, f_e=1.5))
    bad = dict(W.WATER, i_ev=-1.0)
    with pytest.raises(dpm.DpmError):
        dpm.HostTables([bad], P)
    with pytest.raises(dpm.DpmError):
        dpm.HostTables([dict(W.WATER, rho_de=-1.0)], P)


@pytest.mark.parametrize("m", [0, 2])
def test_photon_and_electron_tables(tabs, m):
    L = O.lib()
    mm = O.material(W.MATERIALS[m])
    pr = O.params(P)
    ph, meta = tabs.get("ph")
    el, _ = tabs.get("el")
    pmol, _ = tabs.get("pmol")
    E = np.geomspace(0.051, 20.5, 300)
    mc = lambda e: L.or_mu_compton(mm, e)
    mp = lambda e: L.or_mu_photo(mm, e, P["c_pe"])
    mt = lambda e: mc(e) + mp(e) + L.or_mu_pair(mm, e)
    check(lin_lookup(ph, meta, m, 0, E), mt, E, meta)
    check(lin_lookup(ph, meta, m, 1, E), lambda e: mc(e) / mt(e), E, meta)
    check(lin_lookup(ph, meta, m, 2, E), lambda e: mp(e) / mt(e), E, meta)
    Ee = np.geomspace(0.2, 20.5, 300)
    e_lo = meta[0]
    check(lin_lookup(el, meta, m, 0, Ee), lambda e: L.or_csda_path(mm, pr, e_lo, e), Ee, meta)
    check(lin_lookup(el, meta, m, 1, Ee), lambda e: L.or_scol(mm, e, P["wcc"]) + L.or_srad(mm, e, P["wcr"]), Ee, meta)
    sig = lambda e: L.or_moller_sigma(mm, e, P["wcc"]) + L.or_brems_sigma(mm, e, P["wcr"])
    check(lin_lookup(el, meta, m, 2, Ee), sig, Ee, meta)
    check(lin_lookup(el, meta, m, 3, Ee), lambda e: L.or_lambda1_inv(mm, e), Ee, meta)
    check(lin_lookup(pmol, meta, m, -1, Ee), lambda e: L.or_moller_sigma(mm, e, P["wcc"]) / sig(e) if sig(e) > 0 else 0,
          Ee, meta)


MATERIALS_DE = [dict(W.WATER, rho_de=1.0), dict(W.LUNG, rho_de=0.3), dict(W.BONE, rho_de=1.85)]


@pytest.mark.parametrize("m", [0, 1, 2])
def test_electron_tables_with_density_effect(m):
    """Materials that give a density for the Sternheimer-Peierls correction:
    the builder's stopping power and range against the oracle's, and the
    correction lowers the stopping power by several per cent at 20 MeV."""
    build_lib.build()
    L = O.lib()
    mm = O.material(MATERIALS_DE[m])
    pr = O.params(P)
    with dpm.HostTables(MATERIALS_DE, P) as t, dpm.HostTables(W.MATERIALS, P) as t0:
        el, meta = t.get("el")
        el0, _ = t0.get("el")
        Ee = np.geomspace(0.2, 20.5, 400)
        S = lambda e: L.or_scol(mm, e, P["wcc"]) + L.or_srad(mm, e, P["wcr"])
        check(lin_lookup(el, meta, m, 1, Ee), S, Ee, meta)
        check(lin_lookup(el, meta, m, 0, Ee), lambda e: L.or_csda_path(mm, pr, meta[0], e), Ee, meta)
        s20, s20_0 = lin_lookup(el, meta, m, 1, np.array([20.0]))[0], lin_lookup(el0, meta, m, 1, np.array([20.0]))[0]
        assert 0.02 < 1 - s20 / s20_0 < 0.2
        # below X0 (T < 0.445 MeV for water) the tables agree
        s03, s03_0 = lin_lookup(el, meta, m, 1, np.array([0.3]))[0], lin_lookup(el0, meta, m, 1, np.array([0.3]))[0]
        assert s03 == pytest.approx(s03_0, rel=1e-6) or m != 0


def samp(tab, meta, E, u):
    ne, lo, hi, nu = int(meta[2]), meta[3], meta[4], int(meta[5])
    y = tab.reshape(ne, nu).astype(np.float64)
    x = (math.log(E) - math.log(lo)) * (ne - 1) / (math.log(hi) - math.log(lo))
    x = min(max(x, 0.0), ne - 1 - 1e-3)
    i = int(x)
    fx = x - i
    yk = u * (nu - 1)
    k = np.minimum(yk.astype(int), nu - 2)
    fy = yk - k
    a = y[i, k] + (y[i, k + 1] - y[i, k]) * fy
    b = y[i + 1, k] + (y[i + 1, k + 1] - y[i + 1, k]) * fy
    return a + (b - a) * fx


U = np.linspace(0.0005, 0.9995, 300)


def quad(f, a, b):
    return integrate.quad(f, a, b, epsabs=0, epsrel=1e-10, limit=200)[0]


def test_sampling_tables(tabs):
    L = O.lib()
    m = O.material(W.WATER)
    kn, km = tabs.get("kn")
    for E in [0.06, 1.0, 6.0, 19.0]:
        eps = np.exp(samp(kn, km, E, U) * -math.log1p(2 * E / MC2))
        assert np.abs(np.array([L.or_kn_cdf(E, e) for e in eps]) - U).max() < 5e-5
    mo, mm = tabs.get("mol")
    for T in [0.45, 5.0, 20.0]:
        ec = P["wcc"] / T
        eps = 1 / (1 / ec - samp(mo, mm, T, U) * (1 / ec - 2))
        tot = L.or_moller_sigma(m, T, P["wcc"])
        F = np.array([quad(lambda w: L.or_moller_dsdw(m, T, w), P["wcc"], e * T) / tot for e in eps])
        assert np.abs(F - U).max() < 4e-4
    br, bm = tabs.get("brem")
    for T in [0.1, 5.0, 20.0]:
        k = np.minimum(P["wcr"] * np.exp(samp(br, bm, T, U) * math.log(T / P["wcr"])), T)
        tot = L.or_brems_sigma(m, T, P["wcr"])
        F = np.array([quad(lambda q: L.or_brems_dsdk(m, T, q), P["wcr"], kk) / tot for kk in k])
        assert np.abs(F - U).max() < 5e-5
    pr, pm = tabs.get("pair")
    for E in [2.0, 6.0, 20.0]:
        kp = E / MC2
        d = math.sqrt(1 - 2 * math.exp(0.5) / kp)
        lo, hi = max(1 / kp, 0.5 * (1 - d)), min(1 - 1 / kp, 0.5 * (1 + d))
        eps = lo + samp(pr, pm, E, U) * (hi - lo)
        f = lambda e: L.or_pair_dsde_shape(kp, e, 1)
        tot = quad(f, lo, hi)
        F = np.array([quad(f, lo, e) / tot for e in eps])
        assert np.abs(F - U).max() < 3e-3
        assert abs((F - U).mean()) < 1e-4  # the interpolation error is symmetric


def test_msc_table(tabs):
    L = O.lib()
    ms, meta = tabs.get("msc")
    x0, x1, n = meta[3], meta[4], int(meta[2])
    for q in [1e-7, 1e-4, 0.01, 0.3, 0.9, 0.9999]:
        x = -math.log1p(-q)
        lg = math.log(-math.expm1(-x)) + x
        t = (lg - x0) * (n - 1) / (x1 - x0)
        i = int(t)
        A = math.exp(ms[i] + (ms[i + 1] - ms[i]) * (t - i))
        assert A == pytest.approx(L.or_msc_A(q), rel=2e-5)


def _sauter_cdf_nu(T, nu):
    """CDF in nu = 1 - cos(theta) of Sauter's photoelectron distribution,
    integrated in cos(theta) from the formula in the polar angle."""
    g = 1 + T / MC2
    b = math.sqrt(1 - 1 / g ** 2)
    f = lambda c: (1 - c * c) / (1 - b * c) ** 4 * (1 + 0.5 * g * (g - 1) * (g - 2) * (1 - b * c))
    a = 1 / b - 1
    pts = [1 - a, 1 - 3 * a] if a < 0.3 else None
    tot = integrate.quad(f, -1, 1, epsabs=0, epsrel=1e-11, limit=400, points=pts)[0]
    return np.array([integrate.quad(f, 1 - x, 1, epsabs=0, epsrel=1e-10, limit=400)[0] / tot for x in nu])


def test_sauter_table(tabs):
    """The Sauter table (x / x_max of nu/(A+nu) against u, built from the
    density in x) inverts the distribution written in theta: at the sampled
    nu the CDF returns u within the bilinear interpolation error."""
    sa, sm = tabs.get("sauter")
    assert sm[3] == pytest.approx(P["eabs_e"])
    for T in [0.21, 0.5, 1.5, 6.0, 19.0]:
        g = 1 + T / MC2
        A = 1 / math.sqrt(1 - 1 / g ** 2) - 1
        w = np.arccos(1 - 2 * U) / math.pi  # the table's columns are uniform in w
        x = samp(sa, sm, T, w) * 2 / (2 + A)
        nu = A * x / (1 - x)
        assert nu.min() >= 0 and nu.max() <= 2
        F = _sauter_cdf_nu(T, nu)
        assert np.abs(F - U).max() < 1e-4, (T, np.abs(F - U).max())

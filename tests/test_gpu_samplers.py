"""GPU sampling tables against the oracle's cumulative distributions: the
device maps each uniform u to a value x; the exact FP64 CDF of the model at
x must return u (element-wise, within the interpolation error of the
129-column, 256-row inverse-CDF tables)."""
import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_0910_0329_gb300 import dpm
from paper_0910_0329_gb300 import workloads as W

pytestmark = pytest.mark.gpu
P = W.DEFAULT_PARAMS
MC2 = 0.51099895
U = np.linspace(0.0005, 0.9995, 160)
# Bilinear interpolation on a 256 x 129 grid of a normalised inverse CDF has
# error ~ (1/128)^2/8 * y'' in u plus (dlnE)^2/8 * y'' in energy.  The bounds
# below are about twice the largest error of the host-built tables (measured
# on the CPU, tests/test_host_tables.py): KN 2e-5, brems 3e-5, Moller 3e-4
# (rows at 20 MeV), pair 2e-3 (the density vanishes at the ends of its
# support, so the inverse CDF is steep there), MSC 2e-6.
TOL = {"kn": 1e-4, "mol": 6e-4, "brem": 1e-4, "pair": 4e-3, "msc": 1e-5}


def quad(f, a, b):
    return integrate.quad(f, a, b, epsabs=0, epsrel=1e-10, limit=200)[0]


@pytest.mark.parametrize("E", [0.06, 0.3, 1.0, 3.3, 6.0, 19.0])
def test_kn(tables_ctx, E):
    L = O.lib()
    x = dpm.dpm_diag_sample(tables_ctx.ctx, 0, E, 0.0, U)
    F = np.array([L.or_kn_cdf(E, e) for e in x])
    assert np.max(np.abs(F - U)) < TOL["kn"]


@pytest.mark.parametrize("T", [0.45, 1.0, 5.0, 20.0])
def test_moller(tables_ctx, T):
    L, m = O.lib(), O.material(W.WATER)
    wcc = P["wcc"]
    x = dpm.dpm_diag_sample(tables_ctx.ctx, 1, T, 0.0, U)
    tot = L.or_moller_sigma(m, T, wcc)
    F = np.array([quad(lambda w: L.or_moller_dsdw(m, T, w), wcc, e * T) / tot for e in x])
    assert np.max(np.abs(F - U)) < TOL["mol"]


@pytest.mark.parametrize("T", [0.1, 0.6, 5.0, 20.0])
def test_brems(tables_ctx, T):
    L, m = O.lib(), O.material(W.WATER)
    wcr = P["wcr"]
    x = dpm.dpm_diag_sample(tables_ctx.ctx, 2, T, 0.0, U)
    tot = L.or_brems_sigma(m, T, wcr)
    F = np.array([quad(lambda k: L.or_brems_dsdk(m, T, k), wcr, k) / tot for k in x])
    assert np.max(np.abs(F - U)) < TOL["brem"]


@pytest.mark.parametrize("E", [1.9, 3.0, 6.0, 20.0])
def test_pair(tables_ctx, E):
    L = O.lib()
    k = E / MC2
    x = dpm.dpm_diag_sample(tables_ctx.ctx, 3, E, 0.0, U)
    disc = np.sqrt(1 - 2 * np.exp(0.5) / k)
    lo, hi = max(1 / k, 0.5 * (1 - disc)), min(1 - 1 / k, 0.5 * (1 + disc))
    f = lambda e: L.or_pair_dsde_shape(k, e, 1)
    tot = quad(f, lo, hi)
    F = np.array([quad(f, lo, e) / tot for e in x])
    assert np.max(np.abs(F - U)) < TOL["pair"]


@pytest.mark.parametrize("q", [1e-6, 1e-3, 0.05, 0.4, 0.9, 0.999])
def test_msc(tables_ctx, q):
    L = O.lib()
    A = L.or_msc_A(q)
    x = dpm.dpm_diag_sample(tables_ctx.ctx, 4, 1.0, q, U)
    F = (1 + A) * x / (x + 2 * A)
    assert np.max(np.abs(F - U)) < TOL["msc"]


def test_spectrum(tables_ctx):
    L = O.lib()
    x = dpm.dpm_diag_sample(tables_ctx.ctx, 5, 0.0, 0.0, U)
    F = np.array([L.or_spectrum_cdf(e) for e in x])
    assert np.max(np.abs(F - U)) < 2e-5

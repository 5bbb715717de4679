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


def test_exponential_path(tables_ctx):
    """The free-path sampler -ln(u) with the hardware logarithm, against FP64
    on the device's own float u: at most 2^-21.41 absolute on [0.5, 1) and 3
    ulp relative below (the documented bounds of the intrinsic), never
    negative."""
    u = np.concatenate([np.linspace(1e-7, 0.9999999, 4001), 1.0 - 2.0 ** -np.arange(1, 25)])
    uf = u.astype(np.float32).astype(np.float64)
    x = dpm.dpm_diag_sample(tables_ctx.ctx, 6, 1.0, 0.0, u)
    ref = -np.log(uf)
    assert np.all(x >= 0.0)
    hi = uf >= 0.5
    assert np.max(np.abs(x[hi] - ref[hi])) <= 2.0 ** -21.41
    assert np.max(np.abs(x[~hi] - ref[~hi]) / ref[~hi]) <= 3 * 2.0 ** -23


@pytest.mark.parametrize("c", [-0.9, 0.0, 0.3, 0.999])
def test_rotation(tables_ctx, c):
    """The direction after a turn by polar cosine c and azimuth 2 pi u, by
    properties that do not depend on the basis the rotation uses: a unit
    vector at cosine c to the old direction, whose components across the old
    direction for two azimuths meet at the azimuths' difference."""
    u = np.linspace(0.0, 0.999, 64)
    for start, d in [(0, np.array([0.36, -0.48, 0.8])), (3, np.array([0.0, 0.0, 1.0]))]:
        nv = np.stack([dpm.dpm_diag_sample(tables_ctx.ctx, 7, c, float(start + k), u) for k in range(3)], axis=1)
        assert np.max(np.abs(np.linalg.norm(nv, axis=1) - 1.0)) < 2e-6
        assert np.max(np.abs(nv @ d - c)) < 4e-6
        perp = nv - np.outer(nv @ d, d)
        s2 = 1.0 - c * c
        phi = 2.0 * np.pi * u.astype(np.float32).astype(np.float64)
        gram = perp @ perp.T
        assert np.max(np.abs(gram - s2 * np.cos(phi[:, None] - phi[None, :]))) < 8e-6
        # increasing azimuth turns right-handed about the old direction
        assert np.dot(np.cross(perp[0], perp[16]), d) == pytest.approx(s2 * np.sin(phi[16] - phi[0]), abs=8e-6)


def test_face_distance(tables_ctx):
    """The path to a voxel face with the hardware division: within 2 ulp of the
    quotient (the intrinsic's documented bound, 4 * 2^-24 relative) plus half
    an ulp for the numerator's rounding, against FP64 on the device's float
    inputs."""
    x = np.linspace(0.0, 0.999, 500)
    xf = x.astype(np.float32).astype(np.float64)
    for c in (1.0, 0.7, 0.05, 1e-4, -0.3):
        got = dpm.dpm_diag_sample(tables_ctx.ctx, 8, c, 0.0, x)
        cf = float(np.float32(c))
        ref = (1.0 - xf) / cf if cf > 0 else (0.0 - xf) / cf
        ref = np.maximum(ref, 0.0)
        assert np.all(got >= 0.0)
        assert np.all(np.abs(got - ref) <= 6 * 2.0 ** -24 * ref + 1e-30), (c, np.max(np.abs(got - ref) / np.maximum(ref, 1e-30)))


def _sauter_cdf_nu(T, nu):
    """CDF in nu = 1 - cos(theta) of Sauter's photoelectron distribution,
    integrated in cos(theta) from the formula in the polar angle."""
    g = 1 + T / MC2
    b = np.sqrt(1 - 1 / g ** 2)
    f = lambda c: (1 - c * c) / (1 - b * c) ** 4 * (1 + 0.5 * g * (g - 1) * (g - 2) * (1 - b * c))
    tot = quad(f, -1, 1)
    return np.array([quad(f, 1 - x, 1) / tot for x in nu])


@pytest.mark.parametrize("T", [0.25, 1.0, 5.0, 19.0])
def test_sauter(tables_ctx, T):
    """The device's Sauter photoelectron angle (table in acos(1 - 2u)/pi,
    FP32) against Sauter's formula integrated in the polar angle: the CDF at
    the sampled 1 - cos(theta) returns u."""
    nu = dpm.dpm_diag_sample(tables_ctx.ctx, 9, T, 0.0, U)
    assert nu.min() >= 0 and nu.max() <= 2 + 1e-6
    F = _sauter_cdf_nu(T, nu)
    assert np.max(np.abs(F - U)) < 2e-4

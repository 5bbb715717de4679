"""Pins of the oracle's transport loop (CPU only): energy conservation,
narrow-beam attenuation, CSDA range and depth-energy profile against an
independent ODE solution, symmetry, history-split invariance and missed beams.
"""
import dataclasses
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import oracle as O
from paper_0910_0329_gb300 import workloads as W

MC2 = 0.51099895
P = W.DEFAULT_PARAMS


def water_slab(nz, d, rho=1.0, nx=1, ny=1):
    return W.slab_phantom(nx, ny, nz, d, [(0, 1e9, W.MAT_WATER, rho)])


def pencil(ph, particle, energy, spectrum=W.SPEC_MONO):
    X, Y, _ = ph.extent
    return W.Source(particle, spectrum, energy, (X / 2, Y / 2, 0.0), sad=100.0, fx=1e-6, fy=1e-6)


@pytest.mark.parametrize("make", [W.c0_electron_wlw, W.c1_photon_wbw])
def test_energy_conservation_per_history(make):
    wl = make()
    n = 150 if wl.source.particle == W.ELECTRON else 3000
    r = O.run(wl.phantom, W.MATERIALS, wl.params, wl.source, n, wl.seed, workers=2)
    st = r.stats
    assert st["max_balance_rel"] < 1e-9
    assert st["emitted"] == pytest.approx(st["deposited"] + st["escaped"] + st["missed"], rel=1e-12)
    assert r.S1.sum() == pytest.approx(st["deposited"], rel=1e-12)


def test_energy_conservation_with_pairs():
    ph = water_slab(40, 0.5, nx=21, ny=21)
    src = pencil(ph, W.PHOTON, 15.0)
    r = O.run(ph, W.MATERIALS, P, src, 3000, 5, workers=2)
    assert r.stats["n_positrons"] > 20
    assert r.stats["max_balance_rel"] < 1e-9


@pytest.mark.parametrize("E", [0.2, 1.0, 6.0])
def test_uncollided_transmission_homogeneous(E):
    ph = water_slab(60, 0.5)
    n = 40000
    k = O.uncollided(ph, W.MATERIALS, P, pencil(ph, W.PHOTON, E), n, 21)
    L = O.lib()
    m = O.material(W.WATER)
    mu = L.or_mu_compton(m, E) + L.or_mu_photo(m, E, P["c_pe"]) + L.or_mu_pair(m, E)
    p = math.exp(-mu * 1.0 * 30.0)
    z = (k - n * p) / math.sqrt(n * p * (1 - p))
    assert abs(z) < 3.5


def test_uncollided_transmission_heterogeneous():
    # water 0-3 cm / bone (1.85) 3-7 cm / lung (0.3) 7-20 cm / water 20-30 cm
    ph = W.slab_phantom(3, 3, 60, 0.5, [(0, 3, W.MAT_WATER, 1.0), (3, 7, W.MAT_BONE, 1.85),
                                        (7, 20, W.MAT_LUNG, 0.3), (20, 1e9, W.MAT_WATER, 1.0)])
    E, n = 3.0, 40000
    k = O.uncollided(ph, W.MATERIALS, P, pencil(ph, W.PHOTON, E), n, 22)
    L = O.lib()

    def mu(md):
        m = O.material(md)
        return L.or_mu_compton(m, E) + L.or_mu_photo(m, E, P["c_pe"]) + L.or_mu_pair(m, E)

    tau = mu(W.WATER) * 1.0 * 3 + mu(W.BONE) * 1.85 * 4 + mu(W.LUNG) * 0.3 * 13 + mu(W.WATER) * 1.0 * 10
    p = math.exp(-tau)
    z = (k - n * p) / math.sqrt(n * p * (1 - p))
    assert abs(z) < 3.5


def test_csda_range_and_depth_energy_profile():
    """No hard events and no deflections: a pencil electron travels straight
    down and deposits, in each 0.2 cm voxel, the CSDA energy loss across it.
    The reference is an independent ODE solution of dT/dz = -rho S(T)."""
    T0, d = 20.0, 0.2
    ph = water_slab(80, d)
    src = pencil(ph, W.ELECTRON, T0)
    r = O.run(ph, W.MATERIALS, P, src, 1, 3, workers=1, flags=O.OR_NO_HARD | O.OR_NO_MSC)
    L = O.lib()
    m = O.material(W.WATER)
    S = lambda T: L.or_scol(m, T, P["wcc"]) + L.or_srad(m, T, P["wcr"])
    # total path length equals the CSDA range from T0 down to the absorption energy
    rng = integrate.quad(lambda T: 1.0 / S(T), P["eabs_e"], T0, epsrel=1e-12, points=[0.4], limit=200)[0]
    assert r.stats["e_path"] == pytest.approx(rng, rel=1e-9)
    sol = integrate.solve_ivp(lambda z, T: [-S(T[0])], (0, rng), [T0], rtol=1e-12, atol=1e-12, dense_output=True,
                              method="DOP853")
    edges = np.arange(0, rng, d)
    Tz = np.array([sol.sol(z)[0] for z in edges] + [P["eabs_e"]])
    expect = Tz[:-1] - Tz[1:]
    expect[-1] += P["eabs_e"]  # the residual energy is absorbed in the last voxel
    got = r.S1[: len(expect)]
    np.testing.assert_allclose(got, expect, rtol=1e-7, atol=1e-9)
    assert r.S1[len(expect):].sum() == 0.0
    assert r.S1.sum() == pytest.approx(T0, rel=1e-12)


def test_lateral_mirror_symmetry():
    """The beam is centred on the middle voxel column, so energy deposited left
    and right of it must agree.  Voxels along one track are correlated, so the
    test uses independent batches of histories (t-test on batch differences)."""
    wl = W.c0_electron_wlw()
    ph = wl.phantom
    diffs, tots = [], []
    for b in range(16):
        r = O.run(ph, W.MATERIALS, wl.params, wl.source, 150, 123, h0=150 * b, workers=4)
        e = r.S1.reshape(ph.nz, ph.ny, ph.nx)
        left, right = e[:, :, : ph.nx // 2].sum(), e[:, :, ph.nx // 2 + 1:].sum()
        diffs.append(left - right)
        tots.append(left + right)
    diffs = np.array(diffs)
    t = diffs.mean() / (diffs.std(ddof=1) / math.sqrt(len(diffs)))
    assert abs(t) < 3.5


def test_history_split_invariance():
    wl = W.c1_photon_wbw()
    a = O.run(wl.phantom, W.MATERIALS, wl.params, wl.source, 600, 4, workers=1)
    b1 = O.run(wl.phantom, W.MATERIALS, wl.params, wl.source, 250, 4, h0=0, workers=1)
    b2 = O.run(wl.phantom, W.MATERIALS, wl.params, wl.source, 350, 4, h0=250, workers=1)
    np.testing.assert_allclose(a.S1, b1.S1 + b2.S1, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(a.S2, b1.S2 + b2.S2, rtol=1e-12, atol=1e-12)


def test_missed_beam_deposits_nothing():
    wl = W.c1_photon_wbw()
    src = dataclasses.replace(wl.source, iso=(-50.0, -50.0, 10.0))
    r = O.run(wl.phantom, W.MATERIALS, wl.params, src, 200, 4, workers=1)
    assert r.S1.sum() == 0.0
    assert r.stats["n_missed"] == 200
    assert r.stats["missed"] == pytest.approx(r.stats["emitted"], rel=1e-12)


def test_field_projection_on_surface():
    """Primary entry points cover the field scaled by SSD/SAD: with a 10x10 cm
    field at SAD 100 and SSD 90, the dose at the first voxel layer is confined
    to |x - x_c| < 4.5 cm (plus scatter)."""
    wl = W.c1_photon_wbw()
    ph = wl.phantom
    src = dataclasses.replace(wl.source, particle=W.ELECTRON, spectrum=W.SPEC_MONO, energy=1.0)
    r = O.run(ph, W.MATERIALS, wl.params, src, 2000, 8, workers=2, flags=O.OR_NO_MSC | O.OR_NO_HARD)
    d0 = r.S1.reshape(ph.nz, ph.ny, ph.nx)[0]
    xc = (np.arange(ph.nx) + 0.5) * ph.dx - ph.nx * ph.dx / 2
    inside = np.abs(xc) < 4.5 + 0.5
    assert d0[:, ~inside].sum() == 0.0
    assert d0[np.ix_(np.abs(xc) < 4.0, np.abs(xc) < 4.0)].min() > 0


MATERIALS_DE = [dict(W.WATER, rho_de=1.0), dict(W.LUNG, rho_de=0.3), dict(W.BONE, rho_de=1.85)]


def test_density_effect_transport_conserves_energy_and_lengthens_ranges():
    """With the density-effect correction (R20) the transport still conserves
    energy per history, and the lower stopping power lengthens the CSDA path
    above X0 while leaving it unchanged below (delta = 0 under 0.445 MeV in
    water)."""
    wl = W.c0_electron_wlw()
    r = O.run(wl.phantom, MATERIALS_DE, wl.params, wl.source, 150, wl.seed, workers=2)
    assert r.stats["max_balance_rel"] < 1e-9
    L = O.lib()
    pr = O.params(P)
    w, w0 = O.material(MATERIALS_DE[0]), O.material(W.WATER)
    assert L.or_csda_path(w, pr, 0.2, 0.44) == pytest.approx(L.or_csda_path(w0, pr, 0.2, 0.44), rel=1e-12)
    assert L.or_csda_path(w, pr, 0.2, 20.0) > 1.05 * L.or_csda_path(w0, pr, 0.2, 20.0)


def test_plane_second_moments_by_brute_force():
    """The per-plane second moment P2 of a run equals, history by history, the
    square of each history's plane energies (each history run on its own, so
    its S1 is that history's deposits), summed; a one-voxel column (each plane
    one voxel) gives P2 = S2 exactly; and the plane sigma is non-negative."""
    ph = W.slab_phantom(5, 4, 12, 0.4, [(0, 2, W.MAT_WATER, 1.0), (2, 3, W.MAT_BONE, 1.85),
                                        (3, 1e9, W.MAT_LUNG, 0.3)])
    src = dataclasses.replace(pencil(ph, W.ELECTRON, 4.0), fx=1.5, fy=1.2)
    n = 60
    r = O.run(ph, W.MATERIALS, P, src, n, 11, workers=1, planes=True)
    brute = np.zeros(ph.nz)
    for h in range(n):
        one = O.run(ph, W.MATERIALS, P, src, 1, 11, h0=h, workers=1)
        brute += one.S1.reshape(ph.nz, -1).sum(axis=1) ** 2
    assert brute.sum() > 0
    np.testing.assert_allclose(r.P2, brute, rtol=1e-12, atol=1e-300)
    e, s = r.plane_energy_and_sigma(ph.nz)
    np.testing.assert_allclose(e, r.S1.reshape(ph.nz, -1).sum(axis=1) / n, rtol=1e-14)
    assert (s >= 0).all() and s.max() > 0
    col = water_slab(30, 0.2)
    rc = O.run(col, W.MATERIALS, P, pencil(col, W.ELECTRON, 3.0), 40, 3, workers=2, planes=True)
    np.testing.assert_allclose(rc.P2, rc.S2, rtol=1e-12)

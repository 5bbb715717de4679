"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds *inputs only*: material compositions, cut-off parameters,
voxel phantoms and beam descriptions.  It contains none of the transport
arithmetic (no cross sections, no sampling, no tallies), so both the oracle and
the GPU library can take their inputs from here without sharing any part of the
method.

Workloads follow the paper's test problems (Sec. 3): a point source above a
slab phantom of water with a lung or bone insert, with absorption energies of
200 keV for electrons and 50 keV for photons, plus larger seeded "blob"
phantoms with the same three tissue classes.

Phantom layout: ``mat`` (uint8 material index) and ``rho`` (float32 mass
density, g/cm^3) are flat arrays indexed by ``v = i + nx*(j + ny*k)``; the
phantom occupies ``[0, nx*dx] x [0, ny*dy] x [0, nz*dz]`` (cm) and the beam
enters through the plane ``z = 0``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# ---------------------------------------------------------------------------
# Materials: element lists (Z, A in g/mol, mass fraction) and mean excitation
# energy I.  Lung has water's composition (only the density differs).  Bone is
# a single pseudo-element with Z = 13.8 and Z/A = 0.5148 (cortical bone).
# ---------------------------------------------------------------------------
_W_H = 2 * 1.008 / (2 * 1.008 + 15.999)

WATER = {"name": "water", "elements": [(1.0, 1.008, _W_H), (8.0, 15.999, 1.0 - _W_H)], "i_ev": 75.0}
LUNG = {"name": "lung", "elements": [(1.0, 1.008, _W_H), (8.0, 15.999, 1.0 - _W_H)], "i_ev": 75.0}
BONE = {"name": "bone", "elements": [(13.8, 13.8 / 0.5148, 1.0)], "i_ev": 106.4}

MATERIALS = [WATER, LUNG, BONE]
MAT_WATER, MAT_LUNG, MAT_BONE = 0, 1, 2

# Transport parameters.  c_pe fixes the photoelectric strength: it is the value
# for which the Z^4/E^3 photoelectric coefficient of water equals its
# Klein-Nishina coefficient at 30 keV (a model choice; the paper gives none).
DEFAULT_PARAMS = {
    "eabs_e": 0.200,   # electron absorption energy, MeV (Sec. 3)
    "eabs_g": 0.050,   # photon absorption energy, MeV (Sec. 3)
    "wcc": 0.200,      # Moller hard-collision cut, MeV
    "wcr": 0.050,      # bremsstrahlung hard-emission cut, MeV
    "f_e": 0.05,       # max fractional CSDA energy loss per electron step
    "c_pe": 2.3706979738696062e-08,
    "e_max": 21.0,     # upper end of the tabulated energy range, MeV
    "n_e": 2048,       # energy nodes of the GPU tables
}


# ---------------------------------------------------------------------------
# SplitMix64 (Steele, Lea & Flood 2014) for the phantom generator.
# ---------------------------------------------------------------------------
_M64 = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed: int):
        self.s = seed & _M64

    def next_u64(self) -> int:
        self.s = (self.s + 0x9E3779B97F4A7C15) & _M64
        z = self.s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)


@dataclass
class Phantom:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    mat: np.ndarray  # uint8, flat, v = i + nx*(j + ny*k)
    rho: np.ndarray  # float32, flat
    name: str = ""

    @property
    def n_vox(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def extent(self):
        return (self.nx * self.dx, self.ny * self.dy, self.nz * self.dz)


def slab_phantom(nx, ny, nz, d, slabs, name=""):
    """Phantom of z-slabs.  ``slabs`` is a list of (z0, z1, mat, rho) in cm; a
    voxel takes the slab containing its centre."""
    zc = (np.arange(nz) + 0.5) * d
    mat_z = np.zeros(nz, np.uint8)
    rho_z = np.zeros(nz, np.float32)
    for z0, z1, m, r in slabs:
        sel = (zc >= z0) & (zc < z1)
        mat_z[sel] = m
        rho_z[sel] = r
    if (rho_z <= 0).any():
        raise ValueError("slabs do not cover the phantom")
    mat = np.broadcast_to(mat_z[:, None, None], (nz, ny, nx)).reshape(-1).copy()
    rho = np.broadcast_to(rho_z[:, None, None], (nz, ny, nx)).reshape(-1).copy()
    return Phantom(nx, ny, nz, d, d, d, mat, rho, name)


def blob_phantom(nx, ny, nz, d, seed, rho_lung=0.26, rho_water=1.0, rho_bone=1.85, name=""):
    """Seeded smooth Gaussian-blob density field thresholded into three classes.

    f(r) = sum_k a_k exp(-|r - c_k|^2 / (2 s_k^2)) with 40 blobs per (32 cm)^3
    (scaled by volume), centres uniform in the box, s_k ~ U[1, 3] cm and
    a_k ~ U[-1, 1].  Lung where f < -0.25, bone where f > 0.35, water elsewhere.
    Blobs are truncated at 4 s_k.
    """
    g = SplitMix64(seed)
    X, Y, Z = nx * d, ny * d, nz * d
    K = max(1, int(round(40.0 * X * Y * Z / 32.0 ** 3)))
    f = np.zeros((nz, ny, nx), np.float64)
    xc = (np.arange(nx) + 0.5) * d
    yc = (np.arange(ny) + 0.5) * d
    zc = (np.arange(nz) + 0.5) * d
    for _ in range(K):
        cx, cy, cz = g.uniform() * X, g.uniform() * Y, g.uniform() * Z
        s = 1.0 + 2.0 * g.uniform()
        a = 2.0 * g.uniform() - 1.0
        r = 4.0 * s
        ix = slice(max(0, int((cx - r) / d)), min(nx, int((cx + r) / d) + 1))
        iy = slice(max(0, int((cy - r) / d)), min(ny, int((cy + r) / d) + 1))
        iz = slice(max(0, int((cz - r) / d)), min(nz, int((cz + r) / d) + 1))
        ex = np.exp(-((xc[ix] - cx) ** 2) / (2 * s * s))
        ey = np.exp(-((yc[iy] - cy) ** 2) / (2 * s * s))
        ez = np.exp(-((zc[iz] - cz) ** 2) / (2 * s * s))
        f[iz, iy, ix] += a * ez[:, None, None] * ey[None, :, None] * ex[None, None, :]
    mat = np.full(f.shape, MAT_WATER, np.uint8)
    rho = np.full(f.shape, rho_water, np.float32)
    mat[f < -0.25] = MAT_LUNG
    rho[f < -0.25] = rho_lung
    mat[f > 0.35] = MAT_BONE
    rho[f > 0.35] = rho_bone
    return Phantom(nx, ny, nz, d, d, d, mat.reshape(-1), rho.reshape(-1), name)


# ---------------------------------------------------------------------------
# Beams
# ---------------------------------------------------------------------------
PHOTON, ELECTRON = 0, 1
SPEC_MONO, SPEC_6MV = 0, 1


@dataclass
class Source:
    """Point source at distance ``sad`` from the isocentre ``iso``; the field
    ``fx x fy`` is defined in the plane through the isocentre normal to the
    beam axis.  ``gantry_deg`` rotates the beam about the y axis through the
    isocentre (0 = beam travelling along +z)."""
    particle: int
    spectrum: int
    energy: float
    iso: tuple
    sad: float = 100.0
    fx: float = 10.0
    fy: float = 10.0
    gantry_deg: float = 0.0


def axial_source(ph: Phantom, particle, spectrum, energy, ssd, sad, fx, fy):
    """Beam on the central axis of the phantom, normally incident on z = 0, with
    the source ``ssd`` above the surface and the field defined at ``sad``."""
    X, Y, _ = ph.extent
    return Source(particle, spectrum, energy, (X / 2, Y / 2, sad - ssd), sad, fx, fy, 0.0)


@dataclass
class Workload:
    name: str
    phantom: Phantom
    source: Source
    n_histories: int
    seed: int
    params: dict = field(default_factory=lambda: dict(DEFAULT_PARAMS))


def c0_electron_wlw(n_histories=20000, seed=1):
    """20 MeV electrons, SSD 100 cm, 5x5 cm field, 61x61x60 voxels of 0.5 cm,
    water 0-3 cm / lung (0.3 g/cm^3) 3-10 cm / water."""
    ph = slab_phantom(61, 61, 60, 0.5, [(0, 3, MAT_WATER, 1.0), (3, 10, MAT_LUNG, 0.3), (10, 1e9, MAT_WATER, 1.0)],
                      name="wlw_61x61x60")
    src = axial_source(ph, ELECTRON, SPEC_MONO, 20.0, ssd=100.0, sad=100.0, fx=5.0, fy=5.0)
    return Workload("e20_wlw_61x61x60", ph, src, n_histories, seed)


def c1_photon_wbw(n_histories=10_000_000, seed=2):
    """6 MV synthetic spectrum, SSD 90 cm, 10x10 cm field at SAD 100 cm,
    61x61x60 voxels of 0.5 cm, water 0-3 cm / bone (1.85) 3-7 cm / water."""
    ph = slab_phantom(61, 61, 60, 0.5, [(0, 3, MAT_WATER, 1.0), (3, 7, MAT_BONE, 1.85), (7, 1e9, MAT_WATER, 1.0)],
                      name="wbw_61x61x60")
    src = axial_source(ph, PHOTON, SPEC_6MV, 6.0, ssd=90.0, sad=100.0, fx=10.0, fy=10.0)
    p = dict(DEFAULT_PARAMS)
    p["e_max"] = 6.5
    return Workload("6mv_wbw_61x61x60", ph, src, n_histories, seed, p)


def c2_electron_blob128(n_histories=10_000_000, seed=3, phantom_seed=3):
    """20 MeV electrons, SSD 90 cm, 10x10 cm field, 128^3 voxels of 0.25 cm with
    a seeded blob density field (lung 0.26 / water / bone 1.85)."""
    ph = blob_phantom(128, 128, 128, 0.25, phantom_seed, name="blob128")
    src = axial_source(ph, ELECTRON, SPEC_MONO, 20.0, ssd=90.0, sad=100.0, fx=10.0, fy=10.0)
    return Workload("e20_blob128", ph, src, n_histories, seed)


def paper_slab_phantom(middle):
    """The phantom of the paper's experiments (Sec. 3): 30.5 x 30.5 x 30 cm of
    0.5 x 0.5 x 0.2 cm voxels (61 x 61 x 150), water 0-5 cm, then 5 cm of bone
    (1.85 g/cm^3) or lung (0.3 g/cm^3, density not given in the paper), then
    20 cm of water."""
    nx, ny, nz, dz = 61, 61, 150, 0.2
    zc = (np.arange(nz) + 0.5) * dz
    mid = (zc >= 5.0) & (zc < 10.0)
    m_mid, r_mid = (MAT_BONE, 1.85) if middle == "bone" else (MAT_LUNG, 0.3)
    mat_z = np.where(mid, m_mid, MAT_WATER).astype(np.uint8)
    rho_z = np.where(mid, r_mid, 1.0).astype(np.float32)
    mat = np.broadcast_to(mat_z[:, None, None], (nz, ny, nx)).reshape(-1).copy()
    rho = np.broadcast_to(rho_z[:, None, None], (nz, ny, nx)).reshape(-1).copy()
    return Phantom(nx, ny, nz, 0.5, 0.5, dz, mat, rho, name=f"paper_w{middle[0]}w_61x61x150")


def paper_case(particle, middle, n_histories=None, seed=7):
    """One case of the paper's Table 1: a 20 MeV electron (10^7 histories) or
    6 MV photon (10^9) point source at SSD 90 cm with a 10 x 10 cm field at
    SAD 100 cm, normally incident on the centre of the paper's slab phantom."""
    ph = paper_slab_phantom(middle)
    p = dict(DEFAULT_PARAMS)
    if particle == ELECTRON:
        src = axial_source(ph, ELECTRON, SPEC_MONO, 20.0, ssd=90.0, sad=100.0, fx=10.0, fy=10.0)
        n = n_histories or 10_000_000
        name = f"paper_e20_w{middle[0]}w"
    else:
        src = axial_source(ph, PHOTON, SPEC_6MV, 6.0, ssd=90.0, sad=100.0, fx=10.0, fy=10.0)
        p["e_max"] = 6.5
        n = n_histories or 1_000_000_000
        name = f"paper_6mv_w{middle[0]}w"
    return Workload(name, ph, src, n, seed, p)


WORKLOADS = {
    "e20_wlw_61x61x60": c0_electron_wlw,
    "6mv_wbw_61x61x60": c1_photon_wbw,
    "e20_blob128": c2_electron_blob128,
}


def c3_batch(scale=1.0, n_jobs=64, seed=0):
    """64 jobs for one batched launch: sizes uniform over {64^3, 96^3, 128^3,
    256x256x128} voxels of U[0.2, 0.5] cm with seeded blob densities (phantom
    seed 1000+i); even jobs a synthetic 6 MV beam, odd jobs monoenergetic
    electrons of 6..20 MeV; 10x10 cm field, SSD 90 cm; 10^U[5,7] histories
    (times `scale`); run seed 2000+i.  Returns [(Phantom, Source, n, seed)]."""
    g = SplitMix64(0xC3 + seed)
    sizes = [(64, 64, 64), (96, 96, 96), (128, 128, 128), (256, 256, 128)]
    out = []
    for i in range(n_jobs):
        nx, ny, nz = sizes[min(int(g.uniform() * 4), 3)]
        d = round(0.2 + 0.3 * g.uniform(), 3)
        ph = blob_phantom(nx, ny, nz, d, 1000 + i, name=f"batch{i}_{nx}x{ny}x{nz}")
        if i % 2 == 0:
            src = axial_source(ph, PHOTON, SPEC_6MV, 6.0, ssd=90.0, sad=100.0, fx=10.0, fy=10.0)
        else:
            e = float(6 + min(int(g.uniform() * 15), 14))
            src = axial_source(ph, ELECTRON, SPEC_MONO, e, ssd=90.0, sad=100.0, fx=10.0, fy=10.0)
        n = max(1, int(round(10 ** (5 + 2 * g.uniform()) * scale)))
        out.append((ph, src, n, 2000 + i))
    return out

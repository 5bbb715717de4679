"""ctypes front end of the FP64 reference transport (TEST INFRASTRUCTURE).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The product path (the CUDA library and
its binding) never touches it.

``run()`` splits a history range over worker processes started with the
``spawn`` method (never ``fork``: a pool forked after CUDA was initialised can
hang).  Each history draws from its own RANECU stream keyed by (seed, history
id), so the result does not depend on the split.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SOURCES = [os.path.join(_HERE, "dpm_oracle.c")]

OR_NO_HARD, OR_NO_MSC, OR_NO_SECONDARY_PHOTONS, OR_SAUTER = 1, 2, 4, 8
S_KN, S_MOLLER, S_BREMS, S_PAIR, S_MSC, S_SPECTRUM, S_SAUTER, S_ISO_X, S_ISO_Z = range(9)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(s) for s in _SOURCES + [os.path.join(_HERE, "dpm_oracle.h")])
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp] + _SOURCES + ["-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Material(C.Structure):
    _fields_ = [("n_elem", C.c_int), ("Z", C.c_double * 8), ("A", C.c_double * 8), ("w", C.c_double * 8),
                ("i_ev", C.c_double), ("rho_de", C.c_double)]


class Params(C.Structure):
    _fields_ = [("eabs_e", C.c_double), ("eabs_g", C.c_double), ("wcc", C.c_double), ("wcr", C.c_double),
                ("f_e", C.c_double), ("c_pe", C.c_double), ("flags", C.c_int)]


class PhantomS(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("dx", C.c_double), ("dy", C.c_double),
                ("dz", C.c_double), ("mat", C.POINTER(C.c_uint8)), ("rho", C.POINTER(C.c_float))]


class SourceS(C.Structure):
    _fields_ = [("particle", C.c_int), ("spectrum", C.c_int), ("energy", C.c_double), ("iso", C.c_double * 3),
                ("sad", C.c_double), ("fx", C.c_double), ("fy", C.c_double), ("gantry_deg", C.c_double)]


class Stats(C.Structure):
    _fields_ = [("emitted", C.c_double), ("deposited", C.c_double), ("escaped", C.c_double), ("missed", C.c_double),
                ("max_balance_rel", C.c_double), ("deposited2", C.c_double), ("e_path", C.c_double), ("n_hist", C.c_longlong),
                ("n_missed", C.c_longlong), ("n_e_steps", C.c_longlong), ("n_g_interactions", C.c_longlong),
                ("n_g_voxel_steps", C.c_longlong), ("n_dep", C.c_longlong), ("n_dep_runs", C.c_longlong),
                ("n_sec_e", C.c_longlong), ("n_sec_g", C.c_longlong), ("n_positrons", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        d, i, u64, pd = C.c_double, C.c_int, C.c_uint64, C.POINTER(C.c_double)
        pm = C.POINTER(Material)
        for name, args in [("or_kn_sigma", [d]), ("or_kn_dsde", [d, d]), ("or_kn_cdf", [d, d]),
                           ("or_mu_compton", [pm, d]), ("or_mu_photo", [pm, d, d]), ("or_mu_pair", [pm, d]),
                           ("or_pair_integral", [d, d, d, i]), ("or_pair_dsde_shape", [d, d, i]),
                           ("or_gl_integrate_test", [i, d, d]), ("or_x0", [pm]), ("or_scol", [pm, d, d]),
                           ("or_plasma_energy_ev", [pm]), ("or_density_delta", [pm, d]),
                           ("or_srad", [pm, d, d]), ("or_moller_sigma", [pm, d, d]), ("or_moller_dsdw", [pm, d, d]),
                           ("or_brems_sigma", [pm, d, d]), ("or_brems_dsdk", [pm, d, d]),
                           ("or_lambda1_inv", [pm, d]), ("or_csda_path", [pm, C.POINTER(Params), d, d]),
                           ("or_csda_energy", [pm, C.POINTER(Params), d, d]), ("or_msc_A", [d]),
                           ("or_msc_mean", [d]), ("or_spectrum_cdf", [d])]:
            f = getattr(L, name)
            f.argtypes = args
            f.restype = d
        L.or_sample.argtypes = [i, d, d, pm, u64, u64, pd]
        L.or_sample.restype = None
        L.or_kinematics.argtypes = [i, d, d, d, pd, pd]
        L.or_kinematics.restype = None
        L.or_ranecu_stream.argtypes = [C.c_int32, C.c_int32, i, pd, C.POINTER(C.c_int32)]
        L.or_ranecu_stream.restype = None
        L.or_run.argtypes = [C.POINTER(PhantomS), pm, i, C.POINTER(Params), C.POINTER(SourceS), u64, u64, u64, pd, pd,
                             C.POINTER(Stats)]
        L.or_run.restype = i
        L.or_run_planes.argtypes = [C.POINTER(PhantomS), pm, i, C.POINTER(Params), C.POINTER(SourceS), u64, u64, u64,
                                    pd, pd, pd, C.POINTER(Stats)]
        L.or_run_planes.restype = i
        L.or_uncollided.argtypes = [C.POINTER(PhantomS), pm, i, C.POINTER(Params), C.POINTER(SourceS), u64, u64]
        L.or_uncollided.restype = C.c_longlong
        _lib = L
    return _lib


# --------------------------------------------------------------------------
# marshalling helpers
# --------------------------------------------------------------------------
def material(md: dict) -> Material:
    m = Material()
    els = md["elements"]
    m.n_elem = len(els)
    for k, (Z, A, w) in enumerate(els):
        m.Z[k], m.A[k], m.w[k] = Z, A, w
    m.i_ev = md["i_ev"]
    m.rho_de = md.get("rho_de", 0.0)
    return m


def materials(mds) -> "C.Array":
    arr = (Material * len(mds))()
    for k, md in enumerate(mds):
        arr[k] = material(md)
    return arr


def params(pd: dict, flags: int = 0) -> Params:
    return Params(pd["eabs_e"], pd["eabs_g"], pd["wcc"], pd["wcr"], pd["f_e"], pd["c_pe"], flags)


def source(src) -> SourceS:
    s = SourceS()
    s.particle, s.spectrum, s.energy = src.particle, src.spectrum, src.energy
    for k in range(3):
        s.iso[k] = src.iso[k]
    s.sad, s.fx, s.fy, s.gantry_deg = src.sad, src.fx, src.fy, src.gantry_deg
    return s


def phantom_struct(ph, keep: list) -> PhantomS:
    mat = np.ascontiguousarray(ph.mat, dtype=np.uint8)
    rho = np.ascontiguousarray(ph.rho, dtype=np.float32)
    keep += [mat, rho]
    return PhantomS(ph.nx, ph.ny, ph.nz, ph.dx, ph.dy, ph.dz, mat.ctypes.data_as(C.POINTER(C.c_uint8)),
                    rho.ctypes.data_as(C.POINTER(C.c_float)))


@dataclass
class OracleResult:
    S1: np.ndarray      # sum over histories of the energy per voxel, MeV
    S2: np.ndarray      # sum over histories of its square, MeV^2
    n: int
    stats: dict
    P2: np.ndarray = None  # per z plane: sum over histories of the plane's energy squared (planes=True)

    def plane_energy_and_sigma(self, nz):
        """Mean energy per history deposited in each z plane and its standard
        error, history by history (run with planes=True)."""
        n = self.n
        e = self.S1.reshape(nz, -1).sum(axis=1) / n
        var = np.maximum(self.P2 / n - e * e, 0.0)
        return e, np.sqrt(var / max(n - 1, 1))

    def mean_energy(self):
        return self.S1 / self.n

    def total_energy_and_sigma(self):
        """Mean energy deposited per history in the whole phantom and its
        standard error (history by history)."""
        n = self.n
        m = self.stats["deposited"] / n
        var = max(self.stats["deposited2"] / n - m * m, 0.0)
        return m, math.sqrt(var / max(n - 1, 1))

    def sigma_mean_energy(self):
        """Standard error of the per-history mean energy, history by history."""
        n = self.n
        var = np.maximum(self.S2 / n - (self.S1 / n) ** 2, 0.0)
        return np.sqrt(var / max(n - 1, 1))


def _run_chunk(args):
    ph, mats_d, pd, src, h0, h1, seed, flags, planes = args
    keep = []
    phs = phantom_struct(ph, keep)
    V = ph.n_vox
    S1 = np.zeros(V, np.float64)
    S2 = np.zeros(V, np.float64)
    P2 = np.zeros(ph.nz, np.float64) if planes else None
    st = Stats()
    mats = materials(mats_d)
    dp = C.POINTER(C.c_double)
    rc = lib().or_run_planes(C.byref(phs), mats, len(mats_d), C.byref(params(pd, flags)), C.byref(source(src)),
                             h0, h1, seed, S1.ctypes.data_as(dp), S2.ctypes.data_as(dp),
                             P2.ctypes.data_as(dp) if planes else None, C.byref(st))
    if rc != 0:
        raise RuntimeError(f"oracle run failed with {rc}")
    return S1, S2, P2, st.as_dict()


def run(ph, mats_d, pd, src, n, seed, h0=0, workers=None, flags=0, chunks_per_worker=4,
        planes=False) -> OracleResult:
    """Transport histories [h0, h0+n) and return the per-voxel sums (and,
    with planes=True, the per-z-plane second moments)."""
    if workers is None:
        workers = os.cpu_count() or 1
    workers = max(1, min(workers, n if n > 0 else 1))
    if workers == 1 or n < 64:
        S1, S2, P2, st = _run_chunk((ph, mats_d, pd, src, h0, h0 + n, seed, flags, planes))
        return OracleResult(S1, S2, n, st, P2)
    import multiprocessing as mp
    k = workers * chunks_per_worker
    edges = [h0 + (n * i) // k for i in range(k + 1)]
    jobs = [(ph, mats_d, pd, src, edges[i], edges[i + 1], seed, flags, planes) for i in range(k)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        parts = pool.map(_run_chunk, jobs)
    S1 = np.zeros(ph.n_vox)
    S2 = np.zeros(ph.n_vox)
    P2 = np.zeros(ph.nz) if planes else None
    st = {}
    for s1, s2, p2, d in parts:
        S1 += s1
        S2 += s2
        if planes:
            P2 += p2
        for key, val in d.items():
            if key == "max_balance_rel":
                st[key] = max(st.get(key, 0.0), val)
            else:
                st[key] = st.get(key, 0) + val
    return OracleResult(S1, S2, n, st, P2)


def uncollided(ph, mats_d, pd, src, n, seed) -> int:
    keep = []
    phs = phantom_struct(ph, keep)
    return int(lib().or_uncollided(C.byref(phs), materials(mats_d), len(mats_d), C.byref(params(pd)),
                                   C.byref(source(src)), n, seed))


def kinematics(which, a, b, phi, d_in):
    """One interaction's outgoing particles (or_kinematics): ((E1, d1), (E2, d2))."""
    din = np.ascontiguousarray(d_in, dtype=np.float64)
    out = np.zeros(8)
    lib().or_kinematics(which, a, b, phi, din.ctypes.data_as(C.POINTER(C.c_double)),
                        out.ctypes.data_as(C.POINTER(C.c_double)))
    return (out[0], out[1:4]), (out[4], out[5:8])


def sample(which, a=0.0, b=0.0, n=100000, seed=1) -> np.ndarray:
    out = np.zeros(n, np.float64)
    lib().or_sample(which, a, b, None, n, seed, out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def ranecu_stream(s1, s2, n):
    out = np.zeros(n, np.float64)
    st = (C.c_int32 * 2)()
    lib().or_ranecu_stream(s1, s2, n, out.ctypes.data_as(C.POINTER(C.c_double)), st)
    return out, (st[0], st[1])


def fn(name):
    """Direct access to a physics function of the oracle."""
    return getattr(lib(), name)


def mat_ptr(md):
    m = material(md)
    return C.byref(m), m

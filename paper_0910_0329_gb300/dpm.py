"""Thin ctypes binding of the C ABI in include/dpm.h (argument marshalling only).

The module-level functions carry the ABI's names (``dpm_create``,
``dpm_load_phantom``, ``dpm_build_tables``, ``dpm_run``, ``dpm_read_dose`` ...);
``Dpm`` is a small convenience wrapper around them.  Every step of the
transport runs in the CUDA library; if the library is missing or cannot load,
this module raises -- there is no CPU fallback.  PyTorch is used only to pass a
CUDA stream (``stream=torch.cuda.current_stream()``) or device output tensors.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads as W

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "libdpm.so")

DPM_OK, DPM_EINVAL, DPM_ENOMEM, DPM_ECUDA, DPM_EQUEUE_OVERFLOW, DPM_ETIMEOUT, DPM_ESTATE = 0, -1, -2, -3, -4, -5, -6
DPM_ESTEPCAP = -7
KERNEL_QUEUE, KERNEL_HISTORY, KERNEL_PAPER_F32, KERNEL_PAPER_CAS, KERNEL_HISTORY_F64 = 0, 1, 2, 3, 4
NO_HARD, NO_MSC, SAUTER = 1, 2, 4
_NAMES = {0: "DPM_OK", -1: "DPM_EINVAL", -2: "DPM_ENOMEM", -3: "DPM_ECUDA", -4: "DPM_EQUEUE_OVERFLOW",
          -5: "DPM_ETIMEOUT", -6: "DPM_ESTATE", -7: "DPM_ESTEPCAP"}


class DpmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class dpm_material(C.Structure):
    _fields_ = [("n_elem", C.c_int), ("Z", C.c_double * 8), ("A", C.c_double * 8), ("w", C.c_double * 8),
                ("i_ev", C.c_double), ("rho_de", C.c_double)]


class dpm_table_params(C.Structure):
    _fields_ = [("eabs_e", C.c_double), ("eabs_g", C.c_double), ("wcc", C.c_double), ("wcr", C.c_double),
                ("f_e", C.c_double), ("c_pe", C.c_double), ("e_max", C.c_double), ("n_e", C.c_int)]


class dpm_source(C.Structure):
    _fields_ = [("particle", C.c_int), ("spectrum", C.c_int), ("energy", C.c_double), ("iso", C.c_double * 3),
                ("sad", C.c_double), ("fx", C.c_double), ("fy", C.c_double), ("gantry_deg", C.c_double)]


class dpm_run_opts(C.Structure):
    _fields_ = [("kernel", C.c_int), ("n_batches", C.c_int), ("block_size", C.c_int), ("blocks_per_sm", C.c_int),
                ("queue_log2", C.c_int), ("refill_min", C.c_int), ("timeout_s", C.c_double),
                ("physics_flags", C.c_int), ("queue_limit", C.c_int), ("use_graph", C.c_int),
                ("count_events", C.c_int), ("refill_pause", C.c_int)]


class dpm_job(C.Structure):
    _fields_ = [("phantom_id", C.c_int), ("src", dpm_source), ("first_history", C.c_uint64),
                ("n_histories", C.c_uint64), ("seed", C.c_uint64)]


class dpm_serve_opts(C.Structure):
    _fields_ = [("target_rel_sigma", C.c_double), ("first_chunk", C.c_uint64), ("max_chunk", C.c_uint64),
                ("overshoot", C.c_double), ("round_budget", C.c_uint64), ("n_batches", C.c_int),
                ("max_active", C.c_int), ("adaptive", C.c_int), ("hbm_budget_bytes", C.c_uint64)]


class dpm_request_status(C.Structure):
    _fields_ = [("state", C.c_int), ("slot", C.c_int), ("histories", C.c_uint64), ("rounds", C.c_int),
                ("rel_sigma", C.c_double), ("dose_max", C.c_double), ("dmax_voxel", C.c_int)]


class dpm_server_info(C.Structure):
    _fields_ = [("n_pending", C.c_int), ("n_active", C.c_int), ("n_done", C.c_int), ("max_active", C.c_int),
                ("n_rounds", C.c_uint64), ("n_completed", C.c_uint64), ("histories", C.c_uint64),
                ("slot_bytes", C.c_uint64), ("peak_slot_bytes", C.c_uint64), ("gpu_ms", C.c_double)]


REQ_PENDING, REQ_ACTIVE, REQ_DONE, REQ_RELEASED = 0, 1, 2, 3


class dpm_run_stats(C.Structure):
    _fields_ = [("n_histories", C.c_uint64), ("n_batches", C.c_int32), ("error_flags", C.c_int32),
                ("emitted", C.c_double), ("deposited", C.c_double), ("escaped", C.c_double), ("missed", C.c_double),
                ("n_e_steps", C.c_uint64), ("n_g_flights", C.c_uint64), ("n_g_interactions", C.c_uint64),
                ("n_tally_atomics", C.c_uint64), ("n_pushed", C.c_uint64), ("transport_ms", C.c_double),
                ("fold_ms", C.c_double), ("n_transport_launches", C.c_uint64),
                ("n_phase_switches", C.c_uint64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# Every symbol declared in include/dpm.h with its ctypes signature.
_P = C.c_void_p
_SIGS = {
    "dpm_create": (C.c_int, [C.POINTER(_P), C.c_int, C.c_uint64]),
    "dpm_device_bytes": (C.c_int, [_P, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
    "dpm_destroy": (None, [_P]),
    "dpm_last_error": (C.c_char_p, [_P]),
    "dpm_set_stream": (C.c_int, [_P, _P]),
    "dpm_load_phantom": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, C.c_double, _P, _P,
                                   C.POINTER(C.c_int)]),
    "dpm_free_phantom": (C.c_int, [_P, C.c_int]),
    "dpm_update_phantom": (C.c_int, [_P, C.c_int, _P, _P]),
    "dpm_clone_phantom": (C.c_int, [_P, C.c_int, C.POINTER(C.c_int)]),
    "dpm_build_tables": (C.c_int, [_P, C.POINTER(dpm_material), C.c_int, C.POINTER(dpm_table_params)]),
    "dpm_run": (C.c_int, [_P, C.c_int, C.POINTER(dpm_source), C.c_uint64, C.c_uint64, C.c_uint64,
                          C.POINTER(dpm_run_opts)]),
    "dpm_reset_tally": (C.c_int, [_P, C.c_int]),
    "dpm_run_batch": (C.c_int, [_P, _P, C.c_int, C.POINTER(dpm_run_opts)]),
    "dpm_batch_stats": (C.c_int, [_P, C.POINTER(dpm_run_stats)]),
    "dpm_read_dose": (C.c_int, [_P, C.c_int, _P, _P, _P, C.POINTER(dpm_run_stats)]),
    "dpm_read_dose_device": (C.c_int, [_P, C.c_int, _P, _P, C.POINTER(dpm_run_stats)]),
    "dpm_sync": (C.c_int, [_P]),
    "dpm_dmax_sigma": (C.c_int, [_P, _P, C.c_int, _P]),
    "dpm_diag_table": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, _P, _P, _P]),
    "dpm_diag_sample": (C.c_int, [_P, C.c_int, C.c_double, C.c_double, C.c_int, _P, _P]),
    "dpm_diag_philox": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "dpm_diag_l2_peaks": (C.c_int, [_P, C.c_uint64, _P]),
    "dpm_diag_atomic_replay": (C.c_int, [_P, _P, C.c_uint64, C.c_uint64, _P]),
    "dpm_run_noalloc": (C.c_int, [_P, C.c_int, C.POINTER(dpm_source), C.c_uint64, C.c_uint64, C.c_uint64, _P,
                                  C.POINTER(dpm_run_stats)]),
    "dpm_server_create": (C.c_int, [_P, C.POINTER(dpm_serve_opts), C.POINTER(_P)]),
    "dpm_server_destroy": (None, [_P]),
    "dpm_server_submit": (C.c_int, [_P, C.c_int, C.POINTER(dpm_source), C.c_uint64, C.POINTER(C.c_int)]),
    "dpm_server_round": (C.c_int, [_P, C.POINTER(C.c_int)]),
    "dpm_server_status": (C.c_int, [_P, C.c_int, C.POINTER(dpm_request_status)]),
    "dpm_server_info_get": (C.c_int, [_P, C.POINTER(dpm_server_info)]),
    "dpm_server_slot_bytes": (C.c_int, [_P, C.c_int, C.POINTER(C.c_uint64)]),
    "dpm_server_release": (C.c_int, [_P, C.c_int]),
    "dpm_serve_next_chunk": (C.c_uint64, [C.POINTER(dpm_serve_opts), C.c_uint64, C.c_double]),
    "dpm_serve_select": (C.c_int, [_P, C.c_int, C.c_uint64, _P]),
    # include/dpm_host.h (host-only table inspection)
    "dpm_host_tables_build": (_P, [C.POINTER(dpm_material), C.c_int, C.POINTER(dpm_table_params), C.c_char_p]),
    "dpm_host_tables_free": (None, [_P]),
    "dpm_host_tables_get": (C.c_int, [_P, C.c_char_p, _P, C.c_int, _P]),
}

_lib = None


def library_path() -> str:
    return _LIB_PATH


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"CUDA library missing at {_LIB_PATH}; build it with __graft_entry__.build()")
        L = C.CDLL(_LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(ctx, rc):
    if rc != DPM_OK:
        msg = lib().dpm_last_error(ctx).decode() if ctx else ""
        raise DpmError(rc, msg)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_P)


# ---------------------------------------------------------------------------
# ABI-named wrappers
# ---------------------------------------------------------------------------
def dpm_create(device: int = 0, hbm_budget_bytes: int = 0):
    h = _P()
    rc = lib().dpm_create(C.byref(h), device, hbm_budget_bytes)
    _check(None, rc)
    return h


def dpm_device_bytes(ctx):
    """(bytes of device memory the context holds, its budget; 0 = none)."""
    used, budget = C.c_uint64(), C.c_uint64()
    _check(ctx, lib().dpm_device_bytes(ctx, C.byref(used), C.byref(budget)))
    return used.value, budget.value


def dpm_destroy(ctx):
    lib().dpm_destroy(ctx)


def dpm_set_stream(ctx, stream=None):
    """``stream``: a torch.cuda.Stream, a raw cudaStream_t integer, or None."""
    raw = getattr(stream, "cuda_stream", stream)
    _check(ctx, lib().dpm_set_stream(ctx, _P(raw) if raw else None))


def dpm_load_phantom(ctx, ph: W.Phantom) -> int:
    mat = np.ascontiguousarray(ph.mat, np.uint8)
    rho = np.ascontiguousarray(ph.rho, np.float32)
    if mat.size != ph.n_vox or rho.size != ph.n_vox:
        raise ValueError("phantom arrays do not match its shape")
    pid = C.c_int(-1)
    _check(ctx, lib().dpm_load_phantom(ctx, ph.nx, ph.ny, ph.nz, ph.dx, ph.dy, ph.dz, _ptr(mat), _ptr(rho),
                                       C.byref(pid)))
    return pid.value


def dpm_free_phantom(ctx, pid: int):
    _check(ctx, lib().dpm_free_phantom(ctx, pid))


def dpm_clone_phantom(ctx, pid: int) -> int:
    """A device copy of phantom `pid` (same contents and majorant, empty tally)."""
    out = C.c_int(-1)
    _check(ctx, lib().dpm_clone_phantom(ctx, pid, C.byref(out)))
    return out.value


def dpm_update_phantom(ctx, pid: int, ph: W.Phantom):
    """New materials and densities for a loaded phantom of the same size."""
    mat = np.ascontiguousarray(ph.mat, np.uint8)
    rho = np.ascontiguousarray(ph.rho, np.float32)
    _check(ctx, lib().dpm_update_phantom(ctx, pid, _ptr(mat), _ptr(rho)))


def material_struct(md: dict) -> dpm_material:
    m = dpm_material()
    m.n_elem = len(md["elements"])
    for k, (Z, A, w) in enumerate(md["elements"]):
        m.Z[k], m.A[k], m.w[k] = Z, A, w
    m.i_ev = md["i_ev"]
    m.rho_de = md.get("rho_de", 0.0)
    return m


def params_struct(p: dict) -> dpm_table_params:
    return dpm_table_params(p["eabs_e"], p["eabs_g"], p["wcc"], p["wcr"], p["f_e"], p["c_pe"], p["e_max"],
                            int(p["n_e"]))


def dpm_build_tables(ctx, materials, params: dict):
    arr = (dpm_material * len(materials))(*[material_struct(m) for m in materials])
    pp = params_struct(params)
    _check(ctx, lib().dpm_build_tables(ctx, arr, len(materials), C.byref(pp)))


def source_struct(src: W.Source) -> dpm_source:
    s = dpm_source()
    s.particle, s.spectrum, s.energy = src.particle, src.spectrum, src.energy
    for k in range(3):
        s.iso[k] = src.iso[k]
    s.sad, s.fx, s.fy, s.gantry_deg = src.sad, src.fx, src.fy, src.gantry_deg
    return s


def dpm_run(ctx, pid: int, src: W.Source, first: int, n: int, seed: int, opts: dpm_run_opts | None = None):
    s = source_struct(src)
    _check(ctx, lib().dpm_run(ctx, pid, C.byref(s), first, n, seed, C.byref(opts) if opts is not None else None))


def dpm_reset_tally(ctx, pid: int):
    _check(ctx, lib().dpm_reset_tally(ctx, pid))


def dpm_read_dose(ctx, pid: int, n_vox: int, want_dose=True, want_sigma=True, want_raw=True):
    dose = np.zeros(n_vox, np.float64) if want_dose else None
    sigma = np.zeros(n_vox, np.float64) if want_sigma else None
    raw = np.zeros(n_vox, np.int64) if want_raw else None
    st = dpm_run_stats()
    rc = lib().dpm_read_dose(ctx, pid, _ptr(dose) if dose is not None else None,
                             _ptr(sigma) if sigma is not None else None, _ptr(raw) if raw is not None else None,
                             C.byref(st))
    _check(ctx, rc)
    return dose, sigma, raw, st.as_dict()


def dpm_read_dose_device(ctx, pid: int, dose_t, sigma_t):
    """Write dose and sigma into caller-allocated CUDA float64 tensors."""
    st = dpm_run_stats()
    _check(ctx, lib().dpm_read_dose_device(ctx, pid, _P(dose_t.data_ptr()), _P(sigma_t.data_ptr()), C.byref(st)))
    return st.as_dict()


def dpm_dmax_sigma(ctx, pids) -> np.ndarray:
    """[(dose_max Gy/history, sigma, voxel index)] for each phantom id."""
    ids = np.ascontiguousarray(pids, np.int32)
    out = np.zeros((len(ids), 3), np.float64)
    _check(ctx, lib().dpm_dmax_sigma(ctx, _ptr(ids), len(ids), _ptr(out)))
    return out


def dpm_sync(ctx):
    _check(ctx, lib().dpm_sync(ctx))


def dpm_diag_table(ctx, which: int, mat: int, energy, aux=None) -> np.ndarray:
    e = np.ascontiguousarray(energy, np.float64)
    a = np.ascontiguousarray(aux, np.float64) if aux is not None else None
    out = np.zeros(e.size, np.float64)
    _check(ctx, lib().dpm_diag_table(ctx, which, mat, e.size, _ptr(e), _ptr(a) if a is not None else None, _ptr(out)))
    return out


def dpm_diag_sample(ctx, which: int, e: float, aux: float, u) -> np.ndarray:
    uu = np.ascontiguousarray(u, np.float64)
    out = np.zeros(uu.size, np.float64)
    _check(ctx, lib().dpm_diag_sample(ctx, which, e, aux, uu.size, _ptr(uu), _ptr(out)))
    return out


def dpm_diag_philox(ctx, ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, np.uint32).reshape(-1)
    k = np.ascontiguousarray(key, np.uint32).reshape(-1)
    n = c.size // 4
    if k.size != 2 * n:
        raise ValueError("need 4 counter words and 2 key words per block")
    out = np.zeros(4 * n, np.uint32)
    _check(ctx, lib().dpm_diag_philox(ctx, n, _ptr(c), _ptr(k), _ptr(out)))
    return out.reshape(n, 4)


def dpm_diag_l2_peaks(ctx, ws_bytes=16 << 20):
    """(scattered 64-bit atomic adds per second, L2 read bytes per second)
    over an L2-resident buffer of ws_bytes."""
    out = np.zeros(2, np.float64)
    _check(ctx, lib().dpm_diag_l2_peaks(ctx, int(ws_bytes), _ptr(out)))
    return float(out[0]), float(out[1])


def dpm_diag_atomic_replay(ctx, ids, n_vox) -> float:
    """64-bit atomic adds per second for the voxel id stream `ids`."""
    a = np.ascontiguousarray(ids, np.uint32)
    rate = C.c_double(0.0)
    _check(ctx, lib().dpm_diag_atomic_replay(ctx, _ptr(a), a.size, int(n_vox), C.byref(rate)))
    return rate.value


def serve_opts(target=0.01, first_chunk=0, max_chunk=0, overshoot=0.0, round_budget=0, n_batches=0, max_active=0,
               adaptive=1, hbm_budget_bytes=0) -> dpm_serve_opts:
    return dpm_serve_opts(target, first_chunk, max_chunk, overshoot, round_budget, n_batches, max_active, adaptive,
                          hbm_budget_bytes)


class Server:
    """The library's request server (dpm_server_*) on a context."""

    def __init__(self, ctx, opts: dpm_serve_opts):
        self.ctx = ctx
        h = _P()
        _check(ctx, lib().dpm_server_create(ctx, C.byref(opts), C.byref(h)))
        self.h = h

    def _chk(self, rc):
        _check(self.ctx, rc)

    def submit(self, geometry_id, src, seed) -> int:
        rid = C.c_int(-1)
        self._chk(lib().dpm_server_submit(self.h, geometry_id, C.byref(source_struct(src)), seed, C.byref(rid)))
        return rid.value

    def round(self) -> int:
        done = C.c_int(0)
        self._chk(lib().dpm_server_round(self.h, C.byref(done)))
        return done.value

    def status(self, rid) -> dict:
        st = dpm_request_status()
        self._chk(lib().dpm_server_status(self.h, rid, C.byref(st)))
        return {k: getattr(st, k) for k, _ in st._fields_}

    def info(self) -> dict:
        st = dpm_server_info()
        self._chk(lib().dpm_server_info_get(self.h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in st._fields_}

    def slot_bytes(self, geometry_id) -> int:
        b = C.c_uint64()
        self._chk(lib().dpm_server_slot_bytes(self.h, geometry_id, C.byref(b)))
        return b.value

    def release(self, rid):
        self._chk(lib().dpm_server_release(self.h, rid))

    def close(self):
        if self.h:
            lib().dpm_server_destroy(self.h)
            self.h = None


def serve_next_chunk(opts: dpm_serve_opts, histories, rel_sigma) -> int:
    return int(lib().dpm_serve_next_chunk(C.byref(opts), int(histories), float(rel_sigma)))


def serve_select(next_n, budget) -> list:
    a = np.ascontiguousarray(next_n, np.uint64)
    out = np.zeros(max(a.size, 1), np.int32)
    k = lib().dpm_serve_select(_ptr(a), a.size, int(budget), _ptr(out))
    if k < 0:
        raise ValueError("bad arguments")
    return out[:k].tolist()


def run_opts(kernel=KERNEL_QUEUE, n_batches=0, block_size=0, blocks_per_sm=0, queue_log2=0, refill_min=0,
             timeout_s=0.0, physics_flags=0, queue_limit=0, use_graph=0, count_events=0,
             refill_pause=0) -> dpm_run_opts:
    return dpm_run_opts(kernel, n_batches, block_size, blocks_per_sm, queue_log2, refill_min, timeout_s,
                        physics_flags, queue_limit, int(use_graph), int(count_events), int(refill_pause))


def dpm_run_batch(ctx, jobs, opts: dpm_run_opts | None = None):
    """``jobs``: list of (phantom_id, Source, first_history, n_histories, seed)."""
    arr = (dpm_job * max(len(jobs), 1))()
    for k, (pid, src, first, n, seed) in enumerate(jobs):
        arr[k] = dpm_job(pid, source_struct(src), first, n, seed)
    _check(ctx, lib().dpm_run_batch(ctx, arr, len(jobs), C.byref(opts) if opts is not None else None))


def dpm_batch_stats(ctx) -> dict:
    st = dpm_run_stats()
    _check(ctx, lib().dpm_batch_stats(ctx, C.byref(st)))
    return st.as_dict()


class Dpm:
    """Convenience wrapper: one context, tables built from a parameter dict."""

    def __init__(self, device=0, materials=None, params=None, stream=None, hbm_budget_bytes=0):
        self.ctx = dpm_create(device, hbm_budget_bytes)
        if stream is not None:
            dpm_set_stream(self.ctx, stream)
        self.phantoms = {}
        if materials is not None:
            self.build_tables(materials, params or W.DEFAULT_PARAMS)

    def build_tables(self, materials, params):
        dpm_build_tables(self.ctx, materials, params)

    def load_phantom(self, ph: W.Phantom) -> int:
        pid = dpm_load_phantom(self.ctx, ph)
        self.phantoms[pid] = ph
        return pid

    def clone_phantom(self, pid) -> int:
        new = dpm_clone_phantom(self.ctx, pid)
        self.phantoms[new] = self.phantoms[pid]
        return new

    def update_phantom(self, pid, ph: W.Phantom):
        old = self.phantoms[pid]
        if (ph.nx, ph.ny, ph.nz) != (old.nx, old.ny, old.nz):
            raise ValueError("dpm_update_phantom keeps the phantom's dimensions")
        dpm_update_phantom(self.ctx, pid, ph)
        self.phantoms[pid] = ph

    def run(self, pid, src, n, seed, first=0, **opts):
        dpm_run(self.ctx, pid, src, first, n, seed, run_opts(**opts) if opts else None)

    def read(self, pid):
        return dpm_read_dose(self.ctx, pid, self.phantoms[pid].n_vox)

    def reset(self, pid):
        dpm_reset_tally(self.ctx, pid)

    def close(self):
        if self.ctx:
            dpm_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def dpm_load_phantom_raw(ctx, nx, ny, nz, dx, dy, dz, mat_ptr: int, rho_ptr: int) -> int:
    """dpm_load_phantom from raw host pointers (e.g. pinned torch CPU tensors)."""
    pid = C.c_int(-1)
    _check(ctx, lib().dpm_load_phantom(ctx, nx, ny, nz, dx, dy, dz, _P(mat_ptr), _P(rho_ptr), C.byref(pid)))
    return pid.value


class HostTables:
    """The tables as the library builds them, read on the host (no GPU)."""

    def __init__(self, materials, params: dict):
        arr = (dpm_material * len(materials))(*[material_struct(m) for m in materials])
        pp = params_struct(params)
        err = C.create_string_buffer(256)
        self.h = lib().dpm_host_tables_build(arr, len(materials), C.byref(pp), err)
        if not self.h:
            raise DpmError(DPM_EINVAL, err.value.decode())

    def get(self, name: str):
        meta = (C.c_double * 6)()
        n = lib().dpm_host_tables_get(self.h, name.encode(), None, 0, meta)
        if n < 0:
            raise KeyError(name)
        a = np.zeros(n, np.float32)
        lib().dpm_host_tables_get(self.h, name.encode(), _ptr(a), n, meta)
        return a, list(meta)

    def close(self):
        if self.h:
            lib().dpm_host_tables_free(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dpm_run_noalloc(ctx, pid: int, src: W.Source, first: int, n: int, seed: int, d_tally_ptr: int) -> dict:
    """Transport into a caller-owned device int64 tally without allocating
    device memory (the fixed-scratch entry point); ``d_tally_ptr`` is a raw
    device pointer, e.g. ``tensor.data_ptr()`` of a CUDA int64 tensor.
    Returns the run's counters (``deposited`` is NaN: it is the tally's
    increase)."""
    s = source_struct(src)
    st = dpm_run_stats()
    _check(ctx, lib().dpm_run_noalloc(ctx, pid, C.byref(s), first, n, seed, _P(d_tally_ptr), C.byref(st)))
    return st.as_dict()

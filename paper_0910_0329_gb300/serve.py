"""Dose requests that arrive over time, served with continuous batching on one
GPU by the library's server (dpm_server_* in include/dpm.h).

The policies are the library's: each admitted request owns a tally slot (a
device copy of its geometry with its own integer tally) while the slots fit
an HBM budget; every round transports the next chunks of the oldest active
requests that fit the round's history budget in one batched persistent launch
(dpm_run_batch), finds each one's D_max and its sigma on the device
(dpm_dmax_sigma) and retires those that reached the target relative sigma.  A
request's first round transports `chunk` histories; with `adaptive`, a later
round is sized from the request's own relative sigma r after n histories
(about n*(r/target)^2 are needed in all).  Round sizes, history ranges and the
stop decision depend only on the request's own tally, so its result is the
same alone or in any mix.

This module adds what a caller around the library does: it loads each
geometry once (the template its slots copy), submits requests when their
arrival time comes, calls a round while there is work, records arrival,
admission and completion times, reads a finished request's tally if asked and
releases its slot.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import dpm
from . import workloads as W


@dataclass
class Request:
    rid: int
    geometry: int
    source: W.Source
    arrival: float
    # filled in by the server
    admitted: float | None = None
    done: float | None = None
    histories: int = 0
    rounds: int = 0
    rel_sigma: float = math.inf
    dose_max: float = 0.0
    raw: np.ndarray | None = None
    slot: int | None = None

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival


@dataclass
class ServeStats:
    completed: list = field(default_factory=list)
    rounds: int = 0
    histories: int = 0
    wall: float = 0.0
    max_active: int = 0
    peak_bytes: int = 0
    gpu_ms: float = 0.0

    def latencies(self):
        return np.array([r.latency for r in self.completed])

    def summary(self):
        lat = self.latencies()
        return {"requests": len(self.completed), "rounds": self.rounds, "histories": self.histories,
                "wall_s": self.wall, "histories_per_s": self.histories / self.wall if self.wall else 0.0,
                "p50_latency_s": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_latency_s": float(np.percentile(lat, 99)) if len(lat) else None,
                "mean_histories_per_request": self.histories / max(len(self.completed), 1),
                "max_active": self.max_active, "peak_slot_bytes": self.peak_bytes,
                "gpu_busy_frac": self.gpu_ms / 1000.0 / self.wall if self.wall else 0.0}


class Server:
    def __init__(self, geometries, params=None, hbm_budget=16 << 30, chunk=200_000, target=0.01, n_batches=10,
                 max_active=1024, keep_results=False, seed_base=10 ** 6, device=0, stream=None, adaptive=True,
                 max_chunk=None, overshoot=1.15, round_budget=None):
        self.d = dpm.Dpm(device, W.MATERIALS, params or W.DEFAULT_PARAMS, stream=stream)
        self.srv = None
        try:
            self.geoms = list(geometries)
            self.keep = keep_results
            self.seed_base = seed_base
            self.budget = int(hbm_budget)
            # each geometry is resident once: the template its slots copy
            self.template = [self.d.load_phantom(g) for g in self.geoms]
            opts = dict(target=target, first_chunk=int(chunk), max_chunk=int(max_chunk or 0), overshoot=overshoot,
                        round_budget=int(round_budget or 0), n_batches=n_batches, max_active=max_active,
                        adaptive=int(bool(adaptive)))
            probe = dpm.Server(self.d.ctx, dpm.serve_opts(**opts))
            try:
                self.slot_bytes = [probe.slot_bytes(t) for t in self.template]
            finally:
                probe.close()
            # fixed device memory: tables (~1 MB), the queue (an upper bound of
            # its default layout) and the templates; the rest is for slots
            self.fixed = (64 << 20) + 2 * 1216 * (1 << 14) * 13 * 4 + sum(self.slot_bytes)
            if self.budget <= self.fixed:
                raise ValueError(f"hbm_budget {self.budget} is below the fixed {self.fixed} bytes")
            self.srv = dpm.Server(self.d.ctx, dpm.serve_opts(**opts, hbm_budget_bytes=self.budget - self.fixed))
        except BaseException:
            self.d.close()
            raise
        self.stats = ServeStats()

    @property
    def used(self):
        """Device bytes counted against the budget now: fixed part and slots."""
        return self.fixed + self.srv.info()["slot_bytes"]

    def _collect(self, waiting, admitted_by, now):
        """Statuses after a round: admission times, progress, and the done
        requests' results (their slots are released)."""
        for rid in list(waiting):
            r = waiting[rid]
            st = self.srv.status(rid)
            if st["state"] == dpm.REQ_PENDING:
                continue
            if r.admitted is None:
                r.admitted = admitted_by
            r.slot, r.histories, r.rounds = st["slot"], st["histories"], st["rounds"]
            r.rel_sigma, r.dose_max = st["rel_sigma"], st["dose_max"]
            if st["state"] == dpm.REQ_DONE:
                r.done = now
                if self.keep:
                    n_vox = self.geoms[r.geometry].n_vox
                    r.raw = dpm.dpm_read_dose(self.d.ctx, r.slot, n_vox, False, False, True)[2]
                self.srv.release(rid)
                r.slot = None
                self.stats.completed.append(r)
                del waiting[rid]

    def run(self, requests, clock=None, time_scale=1.0):
        """Serve `requests` (sorted by arrival, seconds from start) in real time
        (time_scale > 1 replays arrivals faster).  Returns ServeStats."""
        t0 = time.perf_counter()
        clock = clock or (lambda: (time.perf_counter() - t0) * time_scale)
        base = self.srv.info()
        todo = sorted(requests, key=lambda r: r.arrival)
        waiting = {}  # library request id -> Request
        i = 0
        while i < len(todo) or waiting:
            now = clock()
            while i < len(todo) and todo[i].arrival <= now:
                r = todo[i]
                waiting[self.srv.submit(self.template[r.geometry], r.source, self.seed_base + r.rid)] = r
                i += 1
            if waiting:
                before = self.srv.info()["n_rounds"]
                self.srv.round()
                info = self.srv.info()
                if info["n_rounds"] == before and info["n_pending"]:
                    # nothing active and still nothing admissible, with every
                    # released slot free to go
                    raise RuntimeError("a request does not fit the HBM budget")
                self._collect(waiting, now, clock())
            else:
                time.sleep(max(0.0, (todo[i].arrival - clock()) / time_scale))
        info = self.srv.info()
        self.stats.wall = clock()
        self.stats.rounds += info["n_rounds"] - base["n_rounds"]
        self.stats.histories += info["histories"] - base["histories"]
        self.stats.gpu_ms += info["gpu_ms"] - base["gpu_ms"]
        self.stats.max_active = max(self.stats.max_active, info["max_active"])
        self.stats.peak_bytes = max(self.stats.peak_bytes, self.fixed + info["peak_slot_bytes"])
        return self.stats

    def close(self):
        if self.srv is not None:
            self.srv.close()
            self.srv = None
        self.d.close()


def poisson_requests(n, rate, n_geoms, seed=5, beamlet=0.5, geom_extent=None):
    """n requests with exponential inter-arrival times (rate per second), each
    a 6 MV beamlet of beamlet x beamlet cm at a uniform gantry angle through
    the centre of one of n_geoms geometries (extent (X, Y, Z) per geometry)."""
    g = W.SplitMix64(seed)
    t = 0.0
    out = []
    for r in range(n):
        t += -math.log(max(g.uniform(), 1e-300)) / rate
        k = min(int(g.uniform() * n_geoms), n_geoms - 1)
        theta = 360.0 * g.uniform()
        X, Y, Z = geom_extent[k]
        src = W.Source(W.PHOTON, W.SPEC_6MV, 6.0, (X / 2, Y / 2, Z / 2), 100.0, beamlet, beamlet, theta)
        out.append(Request(r, k, src, t))
    return out

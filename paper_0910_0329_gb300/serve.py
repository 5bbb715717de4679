"""Dose-request server with continuous batching on one GPU.

Requests (a beam on one of the resident phantom geometries) arrive over time.
Each admitted request owns a tally slot (a device copy of its geometry with
its own integer tally); admission is limited by an HBM budget that counts the
tables, the queue memory and every slot.  The server works in rounds: every
round transports the next chunk of histories of all active requests in one
batched persistent launch (dpm_run_batch), then asks the device for each
request's D_max and its sigma (dpm_dmax_sigma) and retires the requests that
reached the target relative uncertainty.  Requests that arrive meanwhile join
at the next round, so work from different requests overlaps on the device.

A request's first round transports `chunk` histories.  With `adaptive`, each
later round is sized from the request's own relative sigma at D_max: with r
after n histories, about n*(r/target)^2 are needed in all, so the next round
transports that (times `overshoot`, within [chunk, max_chunk]) minus n; most
requests then finish in two rounds instead of n_final/chunk.  Without it every
round transports `chunk`.  Round sizes, history ranges (consecutive, with the
request's own seed) and the stop decision depend only on the request's own
tally: its result is the same alone or in any mix.

A round takes the active requests oldest first until their next chunks reach
`round_budget` histories (at least one request).  Under load this keeps the
server close to first-come-first-served -- which minimises the mean latency
of similar requests -- while younger requests fill the round's tail, instead
of advancing every active request together (processor sharing, whose rounds
and latencies grow with the queue).
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
    next_n: int = 0
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
        self.geoms = list(geometries)
        self.chunk = int(chunk)
        self.adaptive = bool(adaptive)
        self.max_chunk = int(max_chunk) if max_chunk else 32 * self.chunk
        self.overshoot = float(overshoot)
        self.round_budget = int(round_budget) if round_budget else 40 * self.chunk
        self.target = float(target)
        self.n_batches = int(n_batches)
        self.max_active = int(max_active)
        self.keep = keep_results
        self.seed_base = seed_base
        self.budget = int(hbm_budget)
        # fixed device memory: tables (~1 MB) and the queue (upper bound of the default layout)
        self.fixed = 64 << 20
        self.fixed += 2 * 1216 * (1 << 14) * 13 * 4
        self.slot_bytes = [g.n_vox * (1 + 4 + 8 + 8 + 8 * self.n_batches) + (512 << 10) for g in self.geoms]
        self.free = {i: [] for i in range(len(self.geoms))}
        self.slot_pid = {}   # slot id -> phantom id
        self.slot_geom = {}
        self.used = self.fixed
        self.pending: list[Request] = []
        self.active: list[Request] = []
        self.stats = ServeStats()

    # -- slots ------------------------------------------------------------
    def _take_slot(self, g):
        if self.free[g]:
            return self.free[g].pop()
        if self.used + self.slot_bytes[g] > self.budget:
            return None
        # a further slot of a geometry already on the device is a device copy
        # (no host scan, upload or wait); the first one is loaded from the host
        same = [pid for pid, gg in self.slot_geom.items() if gg == g]
        pid = self.d.clone_phantom(same[0]) if same else self.d.load_phantom(self.geoms[g])
        self.slot_pid[pid] = pid
        self.slot_geom[pid] = g
        self.used += self.slot_bytes[g]
        self.stats.peak_bytes = max(self.stats.peak_bytes, self.used)
        return pid

    def _release(self, slot):
        dpm.dpm_reset_tally(self.d.ctx, slot)
        self.free[self.slot_geom[slot]].append(slot)

    # -- requests ---------------------------------------------------------
    def submit(self, req: Request):
        self.pending.append(req)

    def _admit(self, now):
        still = []
        for r in self.pending:
            if len(self.active) >= self.max_active:
                still.append(r)
                continue
            slot = self._take_slot(r.geometry)
            if slot is None:
                still.append(r)
                continue
            r.slot = slot
            r.admitted = now
            r.next_n = self.chunk
            self.active.append(r)
        self.pending = still
        self.stats.max_active = max(self.stats.max_active, len(self.active))

    def _round(self, clock):
        chosen = select_round(self.active, self.round_budget)
        jobs = [(r.slot, r.source, r.histories, r.next_n, self.seed_base + r.rid) for r in chosen]
        dpm.dpm_run_batch(self.d.ctx, jobs, dpm.run_opts(n_batches=self.n_batches))
        res = dpm.dpm_dmax_sigma(self.d.ctx, [r.slot for r in chosen])
        # the round's device status (raises on a queue overflow or a timed-out
        # wait) and release of its timing events
        st = dpm.dpm_batch_stats(self.d.ctx)
        self.stats.gpu_ms += st["transport_ms"]
        now = clock()
        self.stats.rounds += 1
        done_ids = set()
        for r, (dose, sig, vox) in zip(chosen, res):
            r.rounds += 1
            r.histories += r.next_n
            self.stats.histories += r.next_n
            r.dose_max = dose
            r.rel_sigma = sig / dose if dose > 0 else math.inf
            r.next_n = self._next_chunk(r)
            if r.rel_sigma <= self.target:
                r.done = now
                if self.keep:
                    r.raw = dpm.dpm_read_dose(self.d.ctx, r.slot, self.geoms[r.geometry].n_vox, False, False, True)[2]
                self._release(r.slot)
                r.slot = None
                self.stats.completed.append(r)
                done_ids.add(r.rid)
        self.active = [r for r in self.active if r.rid not in done_ids]

    def _next_chunk(self, r):
        if not self.adaptive or not math.isfinite(r.rel_sigma) or r.rel_sigma <= 0:
            return self.chunk
        need = r.histories * (r.rel_sigma / self.target) ** 2 * self.overshoot - r.histories
        return int(min(max(need, self.chunk), self.max_chunk))

    def run(self, requests, clock=None, time_scale=1.0):
        """Serve `requests` (sorted by arrival, seconds from start) in real time
        (time_scale > 1 replays arrivals faster).  Returns ServeStats."""
        t0 = time.perf_counter()
        clock = clock or (lambda: (time.perf_counter() - t0) * time_scale)
        todo = sorted(requests, key=lambda r: r.arrival)
        i = 0
        while i < len(todo) or self.pending or self.active:
            now = clock()
            while i < len(todo) and todo[i].arrival <= now:
                self.submit(todo[i])
                i += 1
            self._admit(now)
            if self.active:
                self._round(clock)
            elif i < len(todo):
                time.sleep(max(0.0, (todo[i].arrival - clock()) / time_scale))
            elif self.pending:
                raise RuntimeError("a request does not fit the HBM budget")
        self.stats.wall = clock()
        return self.stats

    def close(self):
        self.d.close()


def select_round(active, budget):
    """The requests of the next round: oldest first (`active` is in arrival
    order), each with its whole next chunk, while the chunks fit in `budget`
    histories; a request that does not fit is passed over for younger ones
    with smaller chunks.  The oldest request always runs."""
    chosen, total = [], 0
    for r in active:
        if chosen and total + r.next_n > budget:
            continue
        chosen.append(r)
        total += r.next_n
    return chosen


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

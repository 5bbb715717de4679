"""Autotuner for the persistent queue launch.

Searches the queue capacity (log2 slots per shard), the resident blocks per SM
and the refill threshold on a short trial of the real workload, by coordinate
descent from the library defaults, and caches the best setting per (GPU,
workload signature) in a JSON file.  The trial runs through the C ABI like any
other run; only the timing source (device time of the transport launches) is
read back.
"""
from __future__ import annotations

import hashlib
import json
import os

DEFAULT_SPACE = {
    "queue_log2": [12, 13, 14, 15],
    "blocks_per_sm": [4, 6, 8],
    "refill_min": [0, 8, 16, 24],  # 0: the library's per-type defaults (24 photon, 12 electron lanes)
}
DEFAULT_START = {"queue_log2": 14, "blocks_per_sm": 8, "refill_min": 0}


def coordinate_descent(trial, space=None, start=None, passes=2, min_gain=0.02):
    """Minimise trial(opts) -> seconds over the grid `space`, one parameter at
    a time, moving only for a gain of at least `min_gain` (so that timing
    noise does not pull the choice away from the start); returns (best_opts,
    best_time, log of (opts, time))."""
    space = space or DEFAULT_SPACE
    start = start or {}
    # start from `start` where it lies in the space, else from the middle value
    best = {k: start[k] if start.get(k) in v else v[len(v) // 2] for k, v in space.items()}
    seen = {}

    def cost(opts):
        key = tuple(sorted(opts.items()))
        if key not in seen:
            seen[key] = trial(dict(opts))
        return seen[key]

    best_t = cost(best)
    for _ in range(passes):
        improved = False
        for name, values in space.items():
            for v in values:
                cand = dict(best, **{name: v})
                t = cost(cand)
                if t < best_t * (1 - min_gain):
                    best, best_t, improved = cand, t, True
        if not improved:
            break
    log = [(dict(k), t) for k, t in seen.items()]
    return best, best_t, log


def signature(gpu_name: str, workload: str) -> str:
    return hashlib.sha256(f"{gpu_name}|{workload}".encode()).hexdigest()[:16]


def default_cache_path() -> str:
    base = os.environ.get("DPM_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "dpm_gb300")
    return os.path.join(base, "autotune.json")


def load(key: str, path: str | None = None):
    path = path or default_cache_path()
    try:
        with open(path) as f:
            return json.load(f).get(key)
    except (OSError, ValueError):
        return None


def save(key: str, entry: dict, path: str | None = None):
    path = path or default_cache_path()
    os.makedirs(os.path.dirname(path), exist_ok=True)
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        data = {}
    data[key] = entry
    tmp = path + f".{os.getpid()}.tmp"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def tune_batch(d, jobs, gpu_name: str, workload: str, fraction=0.25, space=None, use_cache=True, cache_path=None):
    """Tune dpm_run_batch for `jobs` [(pid, src, first, n, seed)] on trials of
    `fraction` of each job's histories; returns the chosen run options dict.
    Trials must be long enough for the kernel's grid-wide phases to switch as
    in the full run (a quarter of the histories by default): on 5 % trials
    the 64-job batch picked options that ran the full batch 4 % slower."""
    from . import dpm

    key = signature(gpu_name, workload)
    if use_cache:
        hit = load(key, cache_path)
        if hit:
            return hit["opts"]
    trial_jobs = [(pid, src, first, max(1000, int(n * fraction)), seed) for pid, src, first, n, seed in jobs]

    def trial(opts):
        dpm.dpm_run_batch(d.ctx, trial_jobs, dpm.run_opts(**opts))
        st = dpm.dpm_batch_stats(d.ctx)
        return st["transport_ms"] / 1000.0

    trial(dict(DEFAULT_START))  # warm-up (allocations, first launch)
    best, t, log = coordinate_descent(trial, space, DEFAULT_START)
    for pid, *_ in jobs:
        dpm.dpm_reset_tally(d.ctx, pid)
    if use_cache:
        save(key, {"opts": best, "trial_s": t, "trials": len(log)}, cache_path)
    return best

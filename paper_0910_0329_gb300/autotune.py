"""Autotuner for the persistent queue launch.

Searches the queue capacity (log2 slots per shard), the resident blocks per SM,
the refill threshold and the refill pause on a short trial of the real
workload, by coordinate descent from the library defaults; the final choice
between the search's best and the defaults is made on full-length runs.  The
result is cached per (GPU, workload signature) in a JSON file.  The trials run
through the C ABI like any other run; only the timing source (device time of
the transport launches) is read back.
"""
from __future__ import annotations

import hashlib
import json
import os

DEFAULT_SPACE = {
    "queue_log2": [12, 13, 14, 15],
    "blocks_per_sm": [4, 6, 8],
    "refill_min": [0, 8, 16, 24],  # 0: the library's per-type defaults (24 photon, 12 electron lanes)
    "refill_pause": [0, -1, 1],  # 0: the library's choice by launch length
}
DEFAULT_START = {"queue_log2": 14, "blocks_per_sm": 8, "refill_min": 0, "refill_pause": 0}


def project(start, space):
    """`start` on the grid `space`: each parameter's start value where the
    space holds it, else the middle of its values."""
    start = start or {}
    return {k: start[k] if start.get(k) in v else v[len(v) // 2] for k, v in space.items()}


def coordinate_descent(trial, space=None, start=None, passes=2, min_gain=0.02):
    """Minimise trial(opts) -> seconds over the grid `space`, one parameter at
    a time, moving only for a gain of at least `min_gain` (so that timing
    noise does not pull the choice away from the start); returns (best_opts,
    best_time, log of (opts, time))."""
    space = space or DEFAULT_SPACE
    best = project(start, space)
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


def confirm(trial_full, best, start, reps=2, min_gain=0.02):
    """The final choice on full-length runs: `best` (found on short trials)
    replaces `start` only if its full run is faster by `min_gain`, each timed
    `reps` times, interleaved, and compared by their minima.  Returns (choice,
    (start time, best time) or None when best is start)."""
    if best == start:
        return dict(start), None
    ts, tb = [], []
    for _ in range(reps):
        ts.append(trial_full(dict(start)))
        tb.append(trial_full(dict(best)))
    t_start, t_best = min(ts), min(tb)
    return (dict(best) if t_best < t_start * (1 - min_gain) else dict(start)), (t_start, t_best)


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
    """Tune dpm_run_batch for `jobs` [(pid, src, first, n, seed)]: search on
    trials of `fraction` of each job's histories, then keep the search's best
    over the defaults only if full-length runs confirm it (short trials
    mislead: on 5 % trials the 64-job batch picked options that ran the full
    batch 4 % slower).  Returns the chosen run options dict."""
    from . import dpm

    key = signature(gpu_name, workload)
    if use_cache:
        hit = load(key, cache_path)
        if hit:
            return hit["opts"]
    trial_jobs = [(pid, src, first, max(1000, int(n * fraction)), seed) for pid, src, first, n, seed in jobs]

    def run(js, opts):
        dpm.dpm_run_batch(d.ctx, js, dpm.run_opts(**opts))
        st = dpm.dpm_batch_stats(d.ctx)
        return st["transport_ms"] / 1000.0

    run(trial_jobs, dict(DEFAULT_START))  # warm-up (allocations, first launch)
    best, t, log = coordinate_descent(lambda o: run(trial_jobs, o), space, DEFAULT_START)
    choice, full = confirm(lambda o: run(jobs, o), best, project(DEFAULT_START, space or DEFAULT_SPACE))
    for pid, *_ in jobs:
        dpm.dpm_reset_tally(d.ctx, pid)
    if use_cache:
        save(key, {"opts": choice, "search_best": best, "trial_s": t, "trials": len(log), "full_s": full},
             cache_path)
    return choice

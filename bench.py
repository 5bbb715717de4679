#!/usr/bin/env python3
"""Throughput benchmark of the coupled electron-photon Monte Carlo transport.

One step = one dpm_run of the whole hot path (source sampling, photon Woodcock
tracking and interactions, condensed-history electron steps, hard events,
fixed-point tally, batch fold) over 10^7 histories of the synthetic 6 MV beam
on the 61x61x60 water/bone/water phantom, with inputs resident on the device.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank transports its own history range on its own
GPU (no data-path collective; weak scaling) and rank 0 prints one JSON line.
``--impl reference`` times the FP64 CPU oracle on the host cores instead
(rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--kernel", choices=["queue", "history", "paper_f32", "paper_cas"], default="queue",
                    help="transport kernel; paper_*: one history per thread with the paper's float tally")
    ap.add_argument("--workload", default="6mv_wbw_61x61x60")
    ap.add_argument("--histories", type=int, default=0, help="histories per step (default: the workload's)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-time-to-target", action="store_true",
                    help="skip the measured time to 1 %% sigma (profiling runs of small steps)")
    ap.add_argument("--cpu-seconds", type=float, default=20.0, help="CPU work of the oracle baseline sample")
    ap.add_argument("--batch-scale", type=float, default=1.0, help="history scale of the batch64 workload")
    ap.add_argument("--autotune", action="store_true", help="tune the batched launch before timing it")
    ap.add_argument("--requests", type=int, default=500, help="requests of the serve workload")
    ap.add_argument("--rate", type=float, default=20.0, help="request arrival rate of the serve workload (1/s)")
    ap.add_argument("--chunk", type=int, default=200000, help="histories of a request's first round (serve)")
    ap.add_argument("--round-budget", type=int, default=0, help="histories per serving round (0: the server's default)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.idx), "-lms", "200"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# --kernel: (dpm_run_opts.kernel, the transport kernel's name)
KERNELS = {"queue": (0, "k_queue"), "history": (1, "k_history"), "paper_f32": (2, "k_history_paper"),
           "paper_cas": (3, "k_history_paper")}


def profiled_traffic(kernel: str, workload: str, key: str = "traffic_bytes_per_history"):
    """Bytes per history of `kernel` (DRAM traffic, or with key
    l2_bytes_per_history the L1->L2 sector traffic) from the committed ncu
    summary, if the kernel's source has not changed since the capture (else
    None)."""
    import re

    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    fp = re.search(r"first 16 hex digits\): `([0-9a-f]{16})`", text)
    tb = re.search(key + r": ([0-9.]+)", text)
    if not fp or not tb:
        return None
    return float(tb.group(1)) if kernel_fingerprint(kernel) == fp.group(1) else None


SM_COUNT, SCHEDULERS_PER_SM = 152, 4


def issue_roofline(kernel: str, workload: str, hist_per_s: float):
    """Instruction-issue view of the kernel: warp instructions per history
    (from the committed ncu capture, if it matches the kernel's source) times
    the measured histories/s, against the issue ceiling of one warp
    instruction per scheduler per cycle at the maximum SM clock."""
    wph = profiled_traffic(kernel, workload, "warp_inst_per_history")
    issue = profiled_traffic(kernel, workload, "issue_active_pct")
    mhz = None
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            mhz = json.load(f).get("sm_max_mhz")
    mhz = mhz or 2070.0
    peak = SM_COUNT * SCHEDULERS_PER_SM * mhz * 1e6
    ach = wph * hist_per_s if wph else None
    return {"achieved": ach, "peak": peak, "unit": "warp instructions/s", "frac": ach / peak if ach else None,
            "warp_inst_per_history": wph, "issue_active_pct_ncu": issue,
            "what": "warp instructions per history (ncu smsp__inst_executed.sum of the committed capture / its "
                    "histories) x histories/s, against 4 issue slots per SM per cycle at the maximum SM clock"}


def time_to_target(d, pid, wl, chunk, kernel, target=0.01, max_chunks=200, adaptive=True, aim=0.97):
    """Run until sigma/D at D_max <= target, from a fresh tally, checking on
    the device after each run (dpm_dmax_sigma).  The first run has `chunk`
    histories.  With `adaptive` each later run is sized from the relative
    sigma r after n histories, as the request server sizes its rounds: about
    n (r / target)^2 are needed in all, so the run aims at `aim` times that
    (a little short, so that a noisy sigma estimate rarely overshoots) minus
    n, and at least chunk / 8; otherwise every run has `chunk` histories.
    Returns the wall time, histories and runs."""
    import torch

    from paper_0910_0329_gb300 import dpm

    dpm.dpm_reset_tally(d.ctx, pid)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    n = 0
    rel = float("inf")
    k = 0
    m = chunk
    for k in range(1, max_chunks + 1):
        d.run(pid, wl.source, m, wl.seed + 7919, first=n, kernel=kernel)
        n += m
        dose, sig, _ = dpm.dpm_dmax_sigma(d.ctx, [pid])[0]
        rel = sig / dose if dose > 0 else float("inf")
        if rel <= target:
            break
        m = chunk
        if adaptive and math.isfinite(rel):
            m = int(min(max(n * (rel / target) ** 2 * aim - n, chunk / 8), 2 ** 31 - 1))
    return {"wall_s": time.perf_counter() - t0, "histories": n, "chunks": k, "sigma_rel": rel,
            "target": target, "chunk": chunk,
            "rule": ("adaptive: first run `chunk`, then n (r/target)^2 * %.2f - n (at least chunk/8)" % aim)
            if adaptive else "fixed chunks"}


def max_over_ranks(x, world, local):
    """The largest of the ranks' values (the job takes as long as its slowest
    rank); x itself on one rank."""
    if world == 1:
        return x
    import torch
    import torch.distributed as tdist

    t = torch.tensor([float(x)], device=f"cuda:{local}")
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def deposit_stream(raw, n, seed=0):
    """n voxel ids drawn independently with probability proportional to the
    integer tally `raw`: a proxy for how often each voxel receives a deposit
    (the hot spots of the dose are the hot spots of the tally atomics)."""
    import numpy as np

    w = np.clip(np.asarray(raw, np.float64), 0, None)
    cdf = np.cumsum(w)
    u = np.random.default_rng(seed).random(n) * cdf[-1]
    return np.minimum(np.searchsorted(cdf, u, side="right"), len(w) - 1).astype(np.uint32)


def kernel_fingerprint(kernel: str = "k_queue"):
    """First 16 hex digits of the sha256 of a transport kernel's sources
    (dpm_device.cuh and dpm_internal.h, with dpm_queue.cu for k_queue or
    dpm_history.cu for the one-history-per-thread kernels) with comments and
    whitespace removed: edits to comments keep a capture valid."""
    import hashlib
    import re

    src = os.path.join(ROOT, "paper_0910_0329_gb300", "csrc")
    h = hashlib.sha256()
    own = "dpm_queue.cu" if kernel == "k_queue" else "dpm_history.cu"
    for f in ("dpm_device.cuh", own, "dpm_internal.h"):
        with open(os.path.join(src, f)) as fh:
            text = fh.read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        h.update("".join(text.split()).encode())
    return h.hexdigest()[:16]


def run_reference(args, rank):
    """The FP64 oracle on the host cores (the reference arm)."""
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_0910_0329_gb300 import workloads as W

    wl = W.WORKLOADS[args.workload](n_histories=1)
    cores = os.cpu_count() or 1
    # calibrate: per-history cost on one core
    t = time.perf_counter()
    O.run(wl.phantom, W.MATERIALS, wl.params, wl.source, 2000, 99, workers=1)
    per_hist = (time.perf_counter() - t) / 2000
    n_step = max(cores * 64, int(cores * 3.0 / per_hist))  # about 3 s of wall time per step
    times = []
    for i in range(args.warmup + args.steps):
        t = time.perf_counter()
        O.run(wl.phantom, W.MATERIALS, wl.params, wl.source, n_step, 1000 + i, workers=cores)
        if i >= args.warmup:
            times.append(time.perf_counter() - t)
    ms = 1000 * statistics.mean(times)
    value = n_step / (ms / 1000)
    line = {"impl": "reference", "metric": "histories/s", "value": value, "unit": "histories/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "histories_per_step": n_step,
                       "program": "FP64 single-thread-per-process oracle (oracle/dpm_oracle.c), RANECU"},
            "cpu_baseline": {"value": value, "unit": "histories/s", "cores": cores, "kind": "oracle",
                             "sample": f"{n_step} histories of {args.workload} per step"},
            "e2e": {"value": value, "unit": "histories/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(args, wl):
    from oracle import oracle as O
    from paper_0910_0329_gb300 import workloads as W

    cores = os.cpu_count() or 1
    t = time.perf_counter()
    O.run(wl.phantom, W.MATERIALS, wl.params, wl.source, 1000, 99, workers=1)
    per_hist = (time.perf_counter() - t) / 1000
    n = max(cores * 64, int(args.cpu_seconds / per_hist))
    t = time.perf_counter()
    O.run(wl.phantom, W.MATERIALS, wl.params, wl.source, n, 7, workers=cores)
    dt = time.perf_counter() - t
    return {"value": n / dt, "unit": "histories/s", "cores": cores, "kind": "oracle",
            "sample": f"{n} histories of {args.workload} (about {args.cpu_seconds:.0f} s of CPU work), "
                      f"{cores} worker processes"}


def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as tdist

        if args.impl == "reference":
            tdist.init_process_group("gloo")
        else:
            import torch

            # each rank's GPU before NCCL picks one for its communicator
            torch.cuda.set_device(local)
            tdist.init_process_group("nccl")
    if args.impl == "reference":
        run_reference(args, rank)
        if world > 1:
            import torch.distributed as tdist

            tdist.destroy_process_group()
        return

    if args.workload == "batch64":
        bench_batch(args, rank, world, local)
        return
    if args.workload == "serve":
        bench_serve(args, rank, world, local)
        return
    if args.workload == "paper_table1":
        bench_paper_table1(args, rank, world, local)
        return

    import numpy as np
    import torch

    from paper_0910_0329_gb300 import build_lib, dpm, sharding
    from paper_0910_0329_gb300 import workloads as W

    build_lib.build()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    wl = W.WORKLOADS[args.workload]()
    n = args.histories or wl.n_histories
    kernel = KERNELS[args.kernel][0]
    ph = wl.phantom
    d = dpm.Dpm(local, W.MATERIALS, wl.params, stream=stream)
    pid = d.load_phantom(ph)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=f"cuda:{local}")

    def step(i):
        first, _ = sharding.history_range(rank, world, i, n)
        d.run(pid, wl.source, n, wl.seed, first=first, kernel=kernel)

    # warm-up
    for i in range(args.warmup):
        step(1000 + i)
    d.read(pid)
    d.reset(pid)
    torch.cuda.synchronize()

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        import torch.distributed as tdist

        tdist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    t_wall = time.perf_counter()
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            flush.fill_(i & 0xFF)  # write 256 MiB (> L2) between steps, outside the step events
            ev[i][0].record(stream)
            step(i)
            ev[i][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    tot_ms = sum(step_ms)
    if world > 1:
        import torch.distributed as tdist

        t = torch.tensor([tot_ms], device=f"cuda:{local}")
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        tot_ms = float(t.item())
        tdist.barrier()
    dose, sigma, raw, st = d.read(pid)
    n_tot = n * args.steps
    value = world * n_tot / (tot_ms / 1000.0)
    # run counters (tally atomics and secondaries for the roofline, energies
    # for the balance): one more step with counting on, after the timed region
    # (the timed steps do not count, see dpm_run_opts.count_events); same
    # histories, same tally
    d.reset(pid)
    d.run(pid, wl.source, n, wl.seed, first=sharding.history_range(rank, world, 0, n)[0], kernel=kernel,
          count_events=1)
    st_cnt = d.read(pid)[3]

    # statistical efficiency: sigma at D_max after n_tot histories -> time to 1 %
    imax = int(np.argmax(dose))
    rel = float(sigma[imax] / dose[imax]) if dose[imax] > 0 else float("nan")
    n_1pct = n_tot * (rel / 0.01) ** 2
    t_1pct = n_1pct / value
    hi = dose > 0.5 * dose.max()
    mean_rel_50 = float(np.mean(sigma[hi] / dose[hi]))

    # roofline of the transport kernel: algorithmic bytes per history are the
    # 8-byte tally atomics, the 44-byte records each secondary is pushed and
    # popped as, and the primary's record
    peak, peak_kind = measured_peaks()
    t_kernel_s = st["transport_ms"] / 1000.0 / max(st["n_transport_launches"], 1)
    hist_per_launch = n
    atom_per_hist = st_cnt["n_tally_atomics"] / n
    sec_per_hist = st_cnt["n_pushed"] / n
    bytes_per_hist = 8 * atom_per_hist + 88 * sec_per_hist + 44
    achieved = bytes_per_hist * hist_per_launch / t_kernel_s / 1e9
    kname = KERNELS[args.kernel][1]
    tph = profiled_traffic(kname, args.workload)
    hbm = {"achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
           "bytes_per_history": bytes_per_hist,
           "what": "algorithmic bytes (8 B per tally atomic, 88 B per queued secondary, 44 B per primary) per "
                   "launch / the launch's event time, against the measured HBM copy bandwidth"}

    # queue init + transport + fold; transport + fold; transport + float rounding + fold
    launches_per_step = {"queue": 3, "history": 2}.get(args.kernel, 3)

    line = {"metric": "histories/s", "value": value, "unit": "histories/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": args.workload, "histories_per_step": n, "phantom": f"{ph.nx}x{ph.ny}x{ph.nz}",
                       "kernel": args.kernel, "l2": "flushed between steps (256 MiB write)",
                       "parallelism": f"{world} replica(s), disjoint history ranges"},
            "time_to_1pct_sigma_at_dmax_s": t_1pct, "sigma_rel_at_dmax": rel, "histories_accumulated": n_tot * world,
            "mean_sigma_rel_above_half_dmax": mean_rel_50,
            "clocks": clk, "gpu_launches": launches_per_step * args.steps,
            "wall_s_timed_region": wall,
            "energy_balance_rel": abs(st_cnt["emitted"] - st_cnt["deposited"] - st_cnt["escaped"] - st_cnt["missed"])
            / st_cnt["emitted"]}

    # L2 roofline: the tally's scattered 64-bit atomics and the L1->L2 sector
    # traffic (per history, from the committed ncu capture) against this GPU's
    # L2 ceilings measured now by dpm_diag_l2_peaks
    atom_pk, l2_pk = dpm.dpm_diag_l2_peaks(d.ctx, 16 << 20)
    atom_rate = atom_per_hist * hist_per_launch / t_kernel_s
    # the tally's own address stream: ids drawn from this run's tally, replayed
    # as 64-bit atomic adds at full occupancy (hot-spot contention included)
    replay_pk = dpm.dpm_diag_atomic_replay(d.ctx, deposit_stream(raw, 1 << 24), ph.n_vox)
    l2_bph = profiled_traffic(kname, args.workload, "l2_bytes_per_history")
    l2_rate = l2_bph * hist_per_launch / t_kernel_s if l2_bph else None
    # headline: the tally-atomic roofline of the scope (achieved tally atomics
    # per second against the replayed ceiling of the same address stream)
    line["roofline"] = {
        "bound": "l2_atomic_replay", "achieved": atom_rate, "peak": replay_pk, "unit": "atomics/s",
        "frac": atom_rate / replay_pk, "traffic": tph * hist_per_launch if tph else None,
        "peak_kind": "measured live (dpm_diag_atomic_replay: 2^24 voxel ids drawn from this run's tally, issued "
                     "as 64-bit atomic adds at full occupancy)",
        "kernel": kname, "kernel_ms_per_launch": t_kernel_s * 1000, "histories_per_launch": hist_per_launch,
        "tally_atomics_per_history": atom_per_hist, "secondaries_per_history": sec_per_hist,
        "kernel_share_of_step": st["transport_ms"] / max(tot_ms, 1e-9),
        "traffic_what": "dram__bytes_read.sum + dram__bytes_write.sum per launch, scaled from the committed ncu "
                        "capture's bytes per history (null if the kernel changed since)",
        "hbm": hbm,
        "issue": issue_roofline(kname, args.workload, value / world),
    }
    line["l2_roofline"] = {
        "atomics": {"achieved": atom_rate, "peak": atom_pk, "unit": "atomics/s", "frac": atom_rate / atom_pk,
                    "what": "tally atomics of the transport kernel vs scattered 64-bit atomics over 16 MiB"},
        "bandwidth": {"achieved": l2_rate / 1e9 if l2_rate else None, "peak": l2_pk / 1e9, "unit": "GB/s",
                      "frac": l2_rate / l2_pk if l2_rate else None, "bytes_per_history": l2_bph,
                      "what": "L1->L2 sectors per history (ncu capture of this kernel) vs L1-bypassing loads "
                              "swept over 16 MiB"},
        "peak_kind": "measured (dpm_diag_l2_peaks, this run)"}

    # time to 1 % sigma at D_max, measured from a fresh tally with a
    # device-side check of sigma/D at D_max after each run: runs sized from
    # sigma as the serving loop sizes its rounds, and (for comparison) runs of
    # the step's histories each
    if not args.no_time_to_target:
        line["time_to_1pct_sigma_at_dmax_measured"] = time_to_target(d, pid, wl, n, kernel)
        line["time_to_1pct_sigma_at_dmax_measured"]["fixed_chunks"] = time_to_target(d, pid, wl, n, kernel,
                                                                                    adaptive=False)

    if not args.no_e2e:
        line["e2e"] = e2e(args, d, wl, n, kernel, local, rank, world)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args, wl)
    d.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as tdist

        tdist.destroy_process_group()


def bench_batch(args, rank, world, local):
    """64 phantoms and beams of uneven size in one persistent launch per step
    (graph-replayed), against the plain path: the same 64 jobs as 64 dpm_run
    calls on the same GPU."""
    import torch

    from paper_0910_0329_gb300 import autotune, build_lib, dpm, sharding
    from paper_0910_0329_gb300 import workloads as W

    build_lib.build()
    torch.cuda.set_device(local)
    stream = torch.cuda.Stream()
    spec = W.c3_batch(scale=args.batch_scale)
    params = dict(W.DEFAULT_PARAMS, e_max=21.0)
    d = dpm.Dpm(local, W.MATERIALS, params, stream=stream)
    pids = [d.load_phantom(ph) for ph, _, _, _ in spec]
    n_step = sum(n for _, _, n, _ in spec)
    opts = {}
    if args.autotune:
        jobs0 = [(pid, src, 0, n, seed) for pid, (ph, src, n, seed) in zip(pids, spec)]
        opts = autotune.tune_batch(d, jobs0, torch.cuda.get_device_name(local), f"batch64x{args.batch_scale}")

    def jobs_for(step):
        out = []
        for pid, (ph, src, n, seed) in zip(pids, spec):
            first, _ = sharding.history_range(rank, world, step, n)
            out.append((pid, src, first, n, seed))
        return out

    ro = dpm.run_opts(use_graph=1, n_batches=10, **opts)
    for i in range(args.warmup):
        dpm.dpm_run_batch(d.ctx, jobs_for(1000 + i), ro)
    dpm.dpm_batch_stats(d.ctx)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as tdist

        tdist.barrier()
    clocks = Clocks(local)
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        ev[i][0].record(stream)
        dpm.dpm_run_batch(d.ctx, jobs_for(i), ro)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    st = dpm.dpm_batch_stats(d.ctx)
    batch_ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    batch_ms = max_over_ranks(batch_ms, world, local)
    # the plain single-run path: the same jobs one dpm_run at a time
    plain = []
    for rep in range(2):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for pid, src, first, n, seed in jobs_for(2000 + rep):
            dpm.dpm_run(d.ctx, pid, src, first, n, seed, dpm.run_opts(n_batches=10, **opts))
        b.record(stream)
        torch.cuda.synchronize()
        plain.append(a.elapsed_time(b))
    plain_ms = min(plain)
    # ceiling of any launch arrangement: every job at the rate it reaches in
    # a long run of its own (at least 4e6 histories, where the launch's
    # start-up and tail are a few % of it); the jobs' histories at those rates
    ideal_ms = 0.0
    for k, (pid, src, first, n, seed) in enumerate(jobs_for(3000)):
        m = max(n, 4_000_000)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        dpm.dpm_run(d.ctx, pid, src, 10 ** 9 + first, m, seed, dpm.run_opts(n_batches=10, **opts))
        b.record(stream)
        torch.cuda.synchronize()
        ideal_ms += a.elapsed_time(b) * n / m
    d.close()
    value = world * n_step / (batch_ms / 1000.0)
    line = {"metric": "histories/s", "value": value, "unit": "histories/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": batch_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch64", "jobs": len(spec), "histories_per_step": n_step,
                       "voxels_total": int(sum(ph.n_vox for ph, *_ in spec)),
                       "launch": "one persistent queue launch per step, CUDA-graph replay (zero -> transport -> fold)",
                       "tuned_opts": opts, "parallelism": f"{world} replica(s)"},
            "single_run_path": {"ms_per_step": plain_ms, "value": world * n_step / (plain_ms / 1000.0),
                                "what": "the same 64 jobs as 64 dpm_run calls"},
            "speedup_vs_single_runs": plain_ms / batch_ms,
            "steady_state_ceiling": {"ms_per_step": ideal_ms, "speedup_vs_single_runs": plain_ms / ideal_ms,
                                     "what": "each job at the rate of a long run of its own (>= 4e6 histories): "
                                             "the gain any arrangement of the launches could reach"},
            "batch_error_flags": st["error_flags"],
            "clocks": clk, "gpu_launches": args.steps * (2 + len(spec))}
    if rank == 0:
        print(json.dumps(line), flush=True)


def bench_serve(args, rank, world, local):
    """Poisson stream of 6 MV beamlet requests (0.5 x 0.5 cm, uniform gantry
    angle) on 8 resident 128^3 blob phantoms of 0.3 cm voxels, each served to
    1 % sigma at D_max with continuous batching; against the plain path that
    serves one request at a time.  Replicas only under torchrun."""
    import torch

    from paper_0910_0329_gb300 import build_lib, serve
    from paper_0910_0329_gb300 import workloads as W

    build_lib.build()
    torch.cuda.set_device(local)
    geoms = [W.blob_phantom(128, 128, 128, 0.3, 100 + k, name=f"patient{k}") for k in range(8)]
    ext = [g.extent for g in geoms]

    def run(max_active, adaptive=True):
        reqs = serve.poisson_requests(args.requests, args.rate, 8, seed=5 + rank, geom_extent=ext)
        s = serve.Server(geoms, hbm_budget=48 << 30, chunk=args.chunk, target=0.01, max_active=max_active,
                         device=local, adaptive=adaptive, round_budget=args.round_budget or None)
        warm = serve.poisson_requests(4, 1000.0, 8, seed=99, geom_extent=ext)
        s.run(warm)  # allocations and first launches
        s.stats = serve.ServeStats()
        clocks = Clocks(local)
        clocks.start()
        st = s.run(reqs)
        clk = clocks.stop()
        s.close()
        return st.summary(), clk

    batched, clk = run(1024)
    plain, _ = run(1)
    fixed, _ = run(1024, adaptive=False)
    wall = max_over_ranks(batched["wall_s"], world, local)
    line = {"metric": "histories/s", "value": world * batched["histories"] / wall, "unit": "histories/s",
            "n_gpus": world, "steps": args.requests, "warmup": 4, "ms_per_step": 1000 * batched["wall_s"] / args.requests,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "serve", "requests": args.requests, "rate_per_s": args.rate,
                       "geometries": "8 x 128^3 x 0.3 cm blob phantoms", "beamlet": "6 MV 0.5x0.5 cm, gantry U[0,360)",
                       "target": "1 % sigma at D_max", "chunk": args.chunk,
                       "rounds": "first round `chunk` histories, later rounds sized from the request's own sigma",
                       "parallelism": f"{world} replica(s)"},
            "p50_latency_s": batched["p50_latency_s"], "p99_latency_s": batched["p99_latency_s"],
            "served": batched, "single_request_path": plain, "fixed_chunk_rounds": fixed, "clocks": clk}
    if rank == 0:
        print(json.dumps(line), flush=True)


# The paper's Table 1 (C1060 GPU vs one 2.27 GHz Xeon core running DPM):
# average relative uncertainty over D > 50 % D_max and the times of the whole
# simulation (initialisation, transfers and transport).
PAPER_TABLE1 = {
    "paper_e20_wlw": {"histories": 10 ** 7, "sigma_rel_pct": 0.65, "t_cpu_s": 470.0, "t_gpu_s": 80.6},
    "paper_e20_wbw": {"histories": 10 ** 7, "sigma_rel_pct": 0.63, "t_cpu_s": 508.0, "t_gpu_s": 101.8},
    "paper_6mv_wlw": {"histories": 10 ** 9, "sigma_rel_pct": 0.52, "t_cpu_s": 5615.0, "t_gpu_s": 845.8},
    "paper_6mv_wbw": {"histories": 10 ** 9, "sigma_rel_pct": 0.46, "t_cpu_s": 6964.0, "t_gpu_s": 1242.3},
}


def bench_paper_table1(args, rank, world, local):
    """The four cases of the paper's experiments (Sec. 3, Table 1) in the
    paper's geometry and history counts, timed like the paper: the whole
    simulation from context creation and table build through phantom upload,
    transport and the read-back of dose and sigma.  Context only: the physics
    data differ from the paper's (closed forms here, DPM's tables there)."""
    import numpy as np
    import torch

    from paper_0910_0329_gb300 import build_lib, dpm
    from paper_0910_0329_gb300 import workloads as W

    build_lib.build()
    torch.cuda.set_device(local)
    with dpm.Dpm(local, W.MATERIALS, W.DEFAULT_PARAMS) as d:  # process-level CUDA start-up, untimed
        d.run(d.load_phantom(W.paper_slab_phantom("lung")), W.paper_case(W.PHOTON, "lung").source, 100000, 1)
        dpm.dpm_sync(d.ctx)
    cases, tot_n, tot_t = [], 0, 0.0
    for particle, middle in [(W.ELECTRON, "lung"), (W.ELECTRON, "bone"), (W.PHOTON, "lung"), (W.PHOTON, "bone")]:
        wl = W.paper_case(particle, middle)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with dpm.Dpm(local, W.MATERIALS, wl.params) as d:
            pid = d.load_phantom(wl.phantom)
            d.run(pid, wl.source, wl.n_histories, wl.seed)
            dose, sigma, raw, st = d.read(pid)
        t = time.perf_counter() - t0
        hi = dose > 0.5 * dose.max()
        rel = float(np.mean(sigma[hi] / dose[hi]))
        ref = PAPER_TABLE1[wl.name]
        cases.append({"case": wl.name, "histories": wl.n_histories, "t_s": t, "transport_s": st["transport_ms"] / 1e3,
                      "sigma_rel_above_half_dmax_pct": 100 * rel, "error_flags": st["error_flags"],
                      "paper": ref, "speedup_vs_paper_gpu": ref["t_gpu_s"] / t,
                      "speedup_vs_paper_cpu": ref["t_cpu_s"] / t})
        tot_n += wl.n_histories
        tot_t += t
    line = {"metric": "histories/s", "value": world * tot_n / tot_t, "unit": "histories/s", "n_gpus": world,
            "steps": 1, "warmup": 1, "ms_per_step": 1000 * tot_t, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "paper_table1", "geometry": "61x61x150 x (0.5x0.5x0.2 cm), 5/5/20 cm slabs",
                       "timing": "whole simulation per case: context, tables, phantom upload, transport, read-back",
                       "parallelism": f"{world} replica(s)"},
            "cases": cases}
    if rank == 0:
        print(json.dumps(line), flush=True)


def e2e(args, d, wl, n, kernel, local, rank=0, world=1):
    """Same metric through the public C ABI with host buffers: every step
    copies the phantom from pinned host memory, transports, and reads dose and
    sigma back into host memory.  Under torchrun each rank runs its own
    history ranges and the job's rate takes the slowest rank's step time."""
    import torch

    from paper_0910_0329_gb300 import dpm

    ph = wl.phantom
    mat = torch.from_numpy(ph.mat).pin_memory()
    rho = torch.from_numpy(ph.rho).pin_memory()
    dose = torch.empty(ph.n_vox, dtype=torch.float64).pin_memory()
    sig = torch.empty(ph.n_vox, dtype=torch.float64).pin_memory()
    s1 = torch.empty(ph.n_vox, dtype=torch.int64).pin_memory()
    L = dpm.lib()
    times = []
    steps = max(3, min(args.steps, 5))
    # the phantom's device buffers are allocated once; every step copies its
    # contents from pinned host memory, transports and reads the results back
    pid = dpm.dpm_load_phantom_raw(d.ctx, ph.nx, ph.ny, ph.nz, ph.dx, ph.dy, ph.dz, mat.data_ptr(), rho.data_ptr())
    for i in range(steps + 1):
        torch.cuda.synchronize()
        t = time.perf_counter()
        rc = L.dpm_update_phantom(d.ctx, pid, mat.data_ptr(), rho.data_ptr())
        if rc:
            raise dpm.DpmError(rc, L.dpm_last_error(d.ctx).decode())
        dpm.dpm_run(d.ctx, pid, wl.source, (i * world + rank) * n, n, wl.seed, dpm.run_opts(kernel=kernel))
        st = dpm.dpm_run_stats()
        rc = L.dpm_read_dose(d.ctx, pid, dose.data_ptr(), sig.data_ptr(), s1.data_ptr(), dpm.C.byref(st))
        if rc:
            raise dpm.DpmError(rc, L.dpm_last_error(d.ctx).decode())
        if i > 0:
            times.append(time.perf_counter() - t)
    dpm.dpm_free_phantom(d.ctx, pid)
    t = max_over_ranks(statistics.mean(times), world, local)
    return {"value": world * n / t, "unit": "histories/s", "h2d_bytes_per_step": world * ph.n_vox * 5,
            "d2h_bytes_per_step": world * (ph.n_vox * (8 + 8 + 8) + dpm.C.sizeof(dpm.dpm_run_stats)),
            "what": "dpm_update_phantom (pinned host mat+rho) + dpm_run + dpm_read_dose (host dose, sigma, raw)"}


if __name__ == "__main__":
    main()

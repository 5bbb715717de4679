"""Host logic of bench.py (no GPU): the kernel source fingerprint that ties a
committed ncu summary to the source it was captured from, and the lookup of
the summary's per-history traffic, which must refuse a stale capture."""
import math
import os
import shutil

import bench
import pytest

SRC = os.path.join(bench.ROOT, "paper_0910_0329_gb300", "csrc")


@pytest.fixture
def tree(tmp_path, monkeypatch):
    """A copy of the transport sources and profiles under a temporary root."""
    csrc = tmp_path / "paper_0910_0329_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for f in ("dpm_device.cuh", "dpm_queue.cu", "dpm_history.cu", "dpm_internal.h"):
        shutil.copy(os.path.join(SRC, f), csrc / f)
    shutil.copytree(os.path.join(bench.ROOT, "profiles"), tmp_path / "profiles")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def test_fingerprint_is_per_kernel_and_ignores_comments(tree):
    q, h = bench.kernel_fingerprint("k_queue"), bench.kernel_fingerprint("k_history")
    assert q != h and len(q) == 16
    dev = tree / "paper_0910_0329_gb300" / "csrc" / "dpm_device.cuh"
    dev.write_text(dev.read_text() + "\n// a comment\n/* another\n one */\n   \n")
    assert bench.kernel_fingerprint("k_queue") == q
    # a change to the history kernel leaves the queue kernel's fingerprint alone
    hist = tree / "paper_0910_0329_gb300" / "csrc" / "dpm_history.cu"
    hist.write_text(hist.read_text() + "\nnamespace { int unused_marker = 1; }\n")
    assert bench.kernel_fingerprint("k_queue") == q and bench.kernel_fingerprint("k_history") != h
    # a code change to the shared physics changes both
    dev.write_text(dev.read_text() + "\nnamespace { int unused_marker2 = 2; }\n")
    assert bench.kernel_fingerprint("k_queue") != q


def test_profiled_traffic_only_for_the_captured_source(tree):
    # the committed summaries match the committed sources
    t = bench.profiled_traffic("k_queue", "6mv_wbw_61x61x60")
    l2 = bench.profiled_traffic("k_queue", "6mv_wbw_61x61x60", "l2_bytes_per_history")
    assert t is not None and 100.0 < t < 400.0 and l2 is not None and l2 > t
    assert bench.profiled_traffic("k_history", "6mv_wbw_61x61x60") is not None
    assert bench.profiled_traffic("k_queue", "no_such_workload") is None
    # a code change makes the capture stale: no traffic is reported
    q = tree / "paper_0910_0329_gb300" / "csrc" / "dpm_queue.cu"
    q.write_text(q.read_text() + "\nnamespace { int unused_marker = 1; }\n")
    assert bench.profiled_traffic("k_queue", "6mv_wbw_61x61x60") is None
    assert bench.profiled_traffic("k_history", "6mv_wbw_61x61x60") is not None


def test_kernel_table_matches_the_binding():
    from paper_0910_0329_gb300 import dpm
    assert bench.KERNELS["queue"][0] == dpm.KERNEL_QUEUE and bench.KERNELS["history"][0] == dpm.KERNEL_HISTORY
    assert bench.KERNELS["paper_f32"][0] == dpm.KERNEL_PAPER_F32
    assert bench.KERNELS["paper_cas"][0] == dpm.KERNEL_PAPER_CAS


def test_max_over_ranks_on_one_rank():
    assert bench.max_over_ranks(3.5, 1, 0) == 3.5


class _FakeSmi:
    """Stands in for the nvidia-smi process: its sampled CSV lines."""

    def __init__(self, text):
        self.text = text

    def terminate(self):
        pass

    def communicate(self, timeout=None):
        return self.text, ""


def test_clock_samples_are_summarised():
    c = bench.Clocks(0)
    c.proc = _FakeSmi("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                      "0, 2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                      "0, 2070, 2070, 1201.5, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                      "garbage line\n"
                      "0, [N/A], 2070, 0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    r = c.stop()
    assert r == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c = bench.Clocks(0)
    c.proc = _FakeSmi("0, 1500, 2070, 700, 0x8, Active, Not Active, Active, Not Active\n")
    assert c.stop()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    c = bench.Clocks(0)  # never started: no nvidia-smi
    assert c.stop()["samples"] == 0


class _FakeDpm:
    """Stand-in for the library in bench.time_to_target: sigma/D at D_max of
    n histories is r1 / sqrt(n), optionally with a fixed relative bias of the
    estimate (the batch estimate of sigma is itself uncertain)."""

    def __init__(self, r1, bias=1.0):
        self.r1, self.bias, self.n, self.runs = r1, bias, 0, []
        self.ctx = object()

    def run(self, pid, src, n, seed, first=0, kernel=0):
        assert first == self.n  # consecutive history ranges
        self.n += n
        self.runs.append(n)


def _patch(monkeypatch, fake):
    from paper_0910_0329_gb300 import dpm

    monkeypatch.setattr(dpm, "dpm_reset_tally", lambda ctx, pid: None)
    monkeypatch.setattr(dpm, "dpm_dmax_sigma",
                        lambda ctx, ids: [(1.0, fake.bias * fake.r1 / fake.n ** 0.5, 0)])


@pytest.mark.parametrize("bias", [1.0, 0.95, 1.1])
def test_time_to_target_sizes_its_runs_from_sigma(monkeypatch, bias):
    """The stop rule: the first run has the step's histories, the next ones
    are sized from sigma (n (r/target)^2 * 0.97 - n, at least a step / 8), and
    it stops at the first check at or below the target: fewer runs than
    fixed chunks, and at most a top-up more histories."""
    import types

    torch = types.SimpleNamespace(cuda=types.SimpleNamespace(synchronize=lambda: None))
    monkeypatch.setitem(__import__("sys").modules, "torch", torch)
    chunk, r1 = 10_000_000, 100.0  # 1 % at 10^8 histories
    need = (bias * r1 / 0.01) ** 2  # histories at which the estimate reaches 1 %
    wl = types.SimpleNamespace(source=None, seed=1)

    fake = _FakeDpm(r1, bias)
    _patch(monkeypatch, fake)
    res = bench.time_to_target(fake, 0, wl, chunk, 0)
    assert res["sigma_rel"] <= 0.01 and res["histories"] == fake.n == sum(fake.runs)
    assert fake.runs[0] == chunk and all(m >= chunk // 8 for m in fake.runs)
    # the sized run aims 3 % short; then top-ups of at least chunk / 8
    assert res["chunks"] <= 2 + math.ceil(0.04 * need / (chunk // 8))
    assert need * (1 - 1e-9) <= fake.n <= need + chunk // 8
    fixed = _FakeDpm(r1, bias)
    _patch(monkeypatch, fixed)
    res_f = bench.time_to_target(fixed, 0, wl, chunk, 0, adaptive=False)
    assert all(m == chunk for m in fixed.runs) and res_f["chunks"] == len(fixed.runs)
    assert res_f["chunks"] > res["chunks"] and fake.n <= fixed.n + chunk // 8

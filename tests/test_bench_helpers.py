"""Host logic of bench.py (no GPU): the kernel source fingerprint that ties a
committed ncu summary to the source it was captured from, and the lookup of
the summary's per-history traffic, which must refuse a stale capture."""
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

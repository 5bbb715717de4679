"""Build the CUDA library in-tree: paper_0910_0329_gb300/_build/libdpm.so.

Each translation unit is compiled for sm_103a in parallel, then linked with
nvcc.  A rebuild happens when any source is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
INC = os.path.join(os.path.dirname(HERE), "include")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libdpm.so")

CU = ["dpm_capi.cu", "dpm_history.cu", "dpm_queue.cu", "dpm_diag.cu", "dpm_noalloc.cu", "dpm_batch.cu", "dpm_serve.cu"]
CPP = ["dpm_tables.cpp", "dpm_host_tables.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# -fmad=false: no implicit FMA contraction, so every kernel computes a particle
# with the same rounding (explicit fmaf() where the code asks for fusion)
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-fmad=false", "-Xcompiler", "-fPIC", "-I" + INC]


def _nvcc():
    for p in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        cand = os.path.join(p, "bin", "nvcc") if p else ""
        if cand and os.path.exists(cand):
            return cand
    return "nvcc"


def _sources():
    deps = [os.path.join(SRC, f) for f in os.listdir(SRC)] + [os.path.join(INC, f) for f in os.listdir(INC)]
    return deps


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not needs_build():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    # one build at a time (ranks of one job may all ask for it): the others
    # wait on the lock and then find the library up to date
    import fcntl

    with open(os.path.join(OUT, ".lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        if not force and not needs_build():
            return LIB
        return _build(verbose)


def _build(verbose: bool) -> str:
    nvcc = _nvcc()
    jobs = []
    for f in CU + CPP:
        obj = os.path.join(OUT, f + ".o")
        jobs.append(([nvcc] + NVCC_FLAGS + ["-c", os.path.join(SRC, f), "-o", obj], obj))

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)

    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        list(ex.map(run, [j[0] for j in jobs]))
    tmp = LIB + f".{os.getpid()}.tmp"
    run([nvcc] + ARCH + ["-shared", "-o", tmp] + [j[1] for j in jobs])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))

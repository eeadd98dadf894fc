"""Compile the CUDA sources under csrc/ into libqcgraph.so, in-tree.

One nvcc per translation unit (run in parallel), then one link.  Only sm_103a
code is generated.  Host code is compiled without floating-point contraction so
that the host-side weight tables are evaluated exactly as written.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libqcgraph.so")
# debug build: every neighbour id a kernel reads is bounds-checked (QC_DEBUG); one
# device error word shared by all translation units, hence relocatable device code
BUILD_DEBUG = os.path.join(HERE, "_build_debug")
LIB_DEBUG = os.path.join(HERE, "libqcgraph_debug.so")
DEBUG_FLAGS = ["-DQC_DEBUG", "-rdc=true"]
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-I", INCLUDE,
                     "-Xcompiler", "-fPIC,-ffp-contract=off,-fno-fast-math,-O2",
                     "-Xptxas", "-warn-spills"]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libqcgraph.so")
    return path


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps() -> list[str]:
    return sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def up_to_date(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None,
          debug: bool = False) -> str:
    """Compile libqcgraph.so (debug: libqcgraph_debug.so, bounds-checked)."""
    lib, build_dir = (LIB_DEBUG, BUILD_DEBUG) if debug else (LIB, BUILD)
    if not force and up_to_date(lib):
        return lib
    os.makedirs(build_dir, exist_ok=True)
    cc = nvcc()
    flags = NVCC_FLAGS + (DEBUG_FLAGS if debug else []) + list(extra_flags or [])
    jobs = []
    for src in sources():
        obj = os.path.join(build_dir, os.path.basename(src)[:-3] + ".o")
        jobs.append((src, obj, [cc] + flags + ["-c", src, "-o", obj]))

    def run(job):
        src, _, cmd = job
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{res.stderr}")
        return res.stderr

    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        logs = list(ex.map(run, jobs))
    if verbose:
        for (src, _, _), log in zip(jobs, logs):
            if log.strip():
                print(f"--- {os.path.basename(src)}\n{log}")
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = ([cc] + ARCH + (["-rdc=true"] if debug else []) + ["-shared", "-o", tmp] + [o for _, o, _ in jobs] +
           ["-lcudart_static", "-lpthread", "-ldl", "-lrt"])
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link of {os.path.basename(lib)} failed:\n{res.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, debug="--debug" in sys.argv))

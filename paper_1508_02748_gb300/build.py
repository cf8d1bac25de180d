"""Builds librewl.so (the CUDA library behind include/rewl.h) for sm_103a.

    python -m paper_1508_02748_gb300.build [--force]

Each .cu file is compiled in parallel with nvcc, then linked into
``paper_1508_02748_gb300/_build/librewl.so`` (in-tree, git-ignored).  Host code
is compiled without floating-point contraction so that the window geometry
is the same on every host architecture; device code uses no FMA contraction
(``--fmad=false``) so that sums and differences round exactly as written.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "librewl.so")
SOURCES = ["rewl_api.cu", "rewl_kernels.cu", "rewl_sweep_tree.cu", "rewl_join.cu", "rewl_noalloc.cu", "rewl_peaks.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librewl")


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "--fmad=false",
                   "-Xcompiler", "-fPIC,-ffp-contract=off,-fno-fast-math",
                   "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    headers = [os.path.join(CSRC, "rewl_internal.cuh"), os.path.join(CSRC, "rewl_tab.cuh"),
               os.path.join(ROOT, "include", "rewl.h"),
               os.path.abspath(__file__)]
    objs = []
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT_DIR, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            cmd = [nvcc()] + _flags() + ["-c", s, "-o", o]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    with ThreadPoolExecutor(max_workers=len(jobs) or 1) as ex:
        for out in ex.map(run, jobs):
            if verbose and out:
                print(out)
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".{os.getpid()}.tmp"
        run([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))

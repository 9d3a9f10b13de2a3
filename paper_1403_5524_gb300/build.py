"""Build the CUDA libraries in-tree for sm_103a (GB300).

``librm.so``   the R-matrix library: every translation unit under ``csrc/``,
               compiled in parallel with nvcc (``-gencode arch=compute_103a,code=sm_103a``)
               and linked into a shared object next to this file.
``librm_checked.so`` the same sources with ``-DRM_CHECKED``: every guarded index of the
               kernels is checked and a violation recorded instead of performed
               (``rm_checked_report``); the tests load it with ``RM_LIBRARY=checked``.
``libpeak.so`` the FP64 pipe peak probe (``probe/fp64_peak.cu``), the measured
               denominator of the FP64 rooflines the benchmark reports.

Nothing here needs a GPU, so it runs on a build host too.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
PROBE = os.path.join(HERE, "probe")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "librm.so")
PEAK_LIB = os.path.join(HERE, "libpeak.so")
CHECKED_LIB = os.path.join(HERE, "librm_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources(folder=CSRC):
    return sorted(os.path.join(folder, f) for f in os.listdir(folder) if f.endswith(".cu"))


def _compile(src: str, extra, tag: str = "") -> str:
    obj = os.path.join(BUILD, tag + os.path.basename(src)[:-3] + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def _link(objs, out: str):
    tmp = out + ".tmp"
    r = subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link of {out} failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)


def build(verbose: bool = False, extra=()) -> str:
    os.makedirs(BUILD, exist_ok=True)
    jobs = ([(s, "", LIB, []) for s in sources()] + [(s, "chk_", CHECKED_LIB, ["-DRM_CHECKED"]) for s in sources()]
            + [(s, "probe_", PEAK_LIB, []) for s in sources(PROBE)])
    # the longest translation units first, so the pool's tail is short
    jobs.sort(key=lambda j: -os.path.getsize(j[0]))
    with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(lambda j: (j[2], _compile(j[0], list(extra) + j[3], j[1])), jobs))
    for lib in (LIB, CHECKED_LIB, PEAK_LIB):
        _link([o for l, o in objs if l == lib], lib)
        if verbose:
            print("built", lib)
    return LIB


if __name__ == "__main__":
    build(verbose=True, extra=sys.argv[1:])

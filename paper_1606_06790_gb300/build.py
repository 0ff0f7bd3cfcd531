"""Builds libidmrg.so in-tree for sm_103a with nvcc (no cmake, no torch).

The translation units compile in parallel; the shared library lands next to
this file.  Used by ``__graft_entry__.build()`` and importable on its own:

    python -m paper_1606_06790_gb300.build
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
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libidmrg.so")
INCLUDE = os.path.join(ROOT, "include")

CU_SOURCES = ["kernels_f64.cu", "kernels_lanczos.cu", "kernels_svd.cu", "kernels_tc.cu", "kernels_obs.cu", "context.cu"]
CXX_SOURCES = ["plan.cpp", "fits.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _run(cmd):
    p = subprocess.run(cmd, capture_output=True, text=True)
    if p.returncode != 0:
        raise RuntimeError("build step failed:\n" + " ".join(cmd) + "\n" + p.stdout + p.stderr)
    return p.stdout + p.stderr


def build(verbose: bool = False) -> str:
    nvcc = _nvcc()
    os.makedirs(OBJ, exist_ok=True)
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]
    jobs = []
    for src in CU_SOURCES:
        out = os.path.join(OBJ, src.replace(".cu", ".o"))
        jobs.append([nvcc, *ARCH, "-lineinfo", *common, "-c", os.path.join(CSRC, src), "-o", out])
    for src in CXX_SOURCES:
        out = os.path.join(OBJ, src.replace(".cpp", ".o"))
        jobs.append([nvcc, *common, "-x", "c++", "-c", os.path.join(CSRC, src), "-o", out])
    with ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        logs = list(ex.map(_run, jobs))
    objs = [j[-1] for j in jobs]
    tmp = LIB + ".tmp"
    logs.append(_run([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]))
    os.replace(tmp, LIB)
    if verbose:
        print("".join(logs))
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))

"""Build libtpe.so (the C-ABI CUDA library) in-tree with nvcc for sm_103a.

Every translation unit is compiled in parallel, then linked into one shared library next to
this file.  Run ``python -m paper_2006_07859_gb300.build`` or call ``build()``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtpe.so")
SOURCES = ["pairs.cu", "solver.cu", "spectral.cu", "api.cu", "peaks.cu", "static_energy.cu", "coarse.cu", "gnn.cu", "pairs_sym.cu", "edges.cu", "ccd.cu", "penalties.cu", "pins.cu", "pairs_df.cu", "coarse_az.cu", "coarse_factor.cu", "pairs_multi.cu", "bh.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags():
    # host code rounds every product and sum separately (no contraction into fma), as the oracle's numpy
    # does: the Barnes-Hut hierarchy's split decisions compare such sums
    return ["-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
            "-Xcompiler", "-ffp-contract=off", "--expt-relaxed-constexpr", "-I", os.path.join(HERE, "..", "include")]


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OBJ, exist_ok=True)
    headers = [os.path.join(CSRC, h) for h in ("tpe_internal.cuh", "pair_device.cuh", "df.cuh", "coarse.cuh")]
    headers.append(os.path.join(HERE, "..", "include", "tpe.h"))
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OBJ, src.replace(".cu", ".o"))
        if force or _stale(o, [s, *headers]):
            jobs.append([nvcc(), *_flags(), "-c", s, "-o", o])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose:
            sys.stderr.write(r.stderr)
        return r

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        list(ex.map(run, jobs))
    objs = [os.path.join(OBJ, s.replace(".cu", ".o")) for s in SOURCES]
    if force or jobs or not os.path.exists(LIB):
        tmp = LIB + f".tmp{os.getpid()}"
        run([nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))

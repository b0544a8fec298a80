"""Build the sm_103a shared library ``libl1line.so`` in-tree.

Each CUDA translation unit is compiled in parallel with nvcc for
``-gencode arch=compute_103a,code=sm_103a`` and the objects are linked into
one shared library next to this file.  No cmake, no torch extension machinery.
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
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libl1line.so")
# the bounds-checked build (L1L_CHECKS=1): the same sources, every kernel index
# checked; l1line.py loads it when L1LINE_LIB names it
LIB_CHECKS = os.path.join(HERE, "libl1line_checks.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["k_prep.cu", "k_pairs.cu", "k_large.cu", "k_exact.cu", "k_reduce.cu", "k_batch.cu", "k_propose.cu",
           "k_path.cu", "k_solpath.cu", "k_probe.cu", "abi.cu"]
# the pair kernels once per (launch shape, kind): (source, object, defines)
SHAPE_UNITS = [("k_pairs_shape.cu", f"k_pairs_s{sh}_p{pk}.o",
                [f"-DL1L_SHAPE={sh}", f"-DL1L_PERSIST={pk}"])
               for sh in range(3) for pk in range(2)]
UNITS = [(src, src.replace(".cu", ".o"), []) for src in SOURCES] + SHAPE_UNITS


def nvcc() -> str:
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def _flags(verbose: bool):
    f = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include")] + ARCH
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _deps_mtime() -> float:
    ts = [os.path.getmtime(os.path.join(CSRC, f)) for f in os.listdir(CSRC)]
    ts.append(os.path.getmtime(os.path.join(ROOT, "include", "l1line.h")))
    ts.append(os.path.getmtime(__file__))
    return max(ts)


def build(force: bool = False, verbose: bool = False, jobs: int | None = None,
          checks: bool = False) -> str:
    lib = LIB_CHECKS if checks else LIB
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime():
        return lib
    bdir = os.path.join(BUILD, "checks") if checks else BUILD
    os.makedirs(bdir, exist_ok=True)
    cc = nvcc()
    extra = ["-DL1L_CHECKS=1"] if checks else []

    def one(unit):
        src, objname, defs = unit
        obj = os.path.join(bdir, objname)
        cmd = [cc, *_flags(verbose), *extra, *defs, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src} {' '.join(defs)}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    # the slowest units first, so that they start before the quick ones
    units = SHAPE_UNITS + [u for u in UNITS if u not in SHAPE_UNITS]
    with cf.ThreadPoolExecutor(max_workers=jobs or min(len(units), os.cpu_count() or 4)) as ex:
        results = list(ex.map(one, units))
    if verbose:
        for _, err in results:
            sys.stderr.write(err)
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *[o for o, _ in results]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                checks="--checks" in sys.argv))

"""Build the CUDA library ``libhard_hydro.so`` for sm_103a with nvcc.

Each element type is its own translation unit; both compile without automatic
FMA contraction (``--fmad=false``) so that rounding is fixed by the source:
FP64 does one IEEE operation per source operation (the oracle's order) and FP32
fuses only where the source calls ``fmaf``.  The translation units compile in
parallel; the library is built in-tree next to this file.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhard_hydro.so")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
          "-Xptxas", "-warn-spills"]
# No automatic FMA contraction anywhere: the FP64 unit then matches the
# oracle's one-rounding-per-operation order, and the FP32 unit fuses exactly
# where the source says fmaf, so every kernel variant rounds identically.
UNITS = {
    "stage_f32.cu": ["--fmad=false"],
    "stage_f64.cu": ["--fmad=false"],
    "weno_f32.cu": ["--fmad=false"],
    "weno_f64.cu": ["--fmad=false"],
    "rad.cu": ["--fmad=false"],
    "fld.cu": [],
    "hard_hydro.cu": [],
    "noalloc.cu": [],
    "batch.cu": [],
}


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhard_hydro.so")


def _sources():
    out = []
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            if f.endswith((".cu", ".cuh", ".h")):
                out.append(os.path.join(d, f))
    return out


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> str:
    """Compile (if sources changed) and return the library path."""
    if not force and not stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    procs = []
    objs = []
    for unit, flags in UNITS.items():
        obj = os.path.join(BUILD, unit.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *COMMON, *flags, *(extra or []), "-c", os.path.join(CSRC, unit), "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((unit, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT,
                                             text=True)))
        objs.append(obj)
    failed = []
    for unit, p in procs:
        out, _ = p.communicate()
        if out and (verbose or p.returncode):
            print(out, file=sys.stderr)
        if p.returncode:
            failed.append(unit)
    if failed:
        raise RuntimeError(f"nvcc failed on {failed}")
    tmp = LIB + ".tmp"
    link = [cc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode:
        print(r.stdout, file=sys.stderr)
        raise RuntimeError("nvcc link of libhard_hydro.so failed")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))

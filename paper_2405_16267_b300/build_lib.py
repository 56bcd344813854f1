"""Build libbicadmm.so in-tree with nvcc for sm_103a (B300).

    python -m paper_2405_16267_b300.build_lib          # build if sources are newer
    python -m paper_2405_16267_b300.build_lib --force  # rebuild
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys
import time

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libbicadmm.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# One whole-unit compilation: splitting the unit across threads (--split-compile) made
# the registers of unchanged kernels depend on unrelated source changes (one x-update kernel
# moved between 32 and 58 registers and ran 38 % slower).
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", "-cudart", "static",
         "-Xptxas", "-O3"]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                  + [os.path.join(INCLUDE, "bicadmm.h")])


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in sources())


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    tmp = "%s.tmp.%d" % (LIB, os.getpid())  # concurrent builds never share a partial file
    cmd = [nvcc(), *ARCH, *FLAGS, "-I", INCLUDE, "-I", CSRC, *extra,
           *sorted(glob.glob(os.path.join(CSRC, "*.cu"))), "-o", tmp]
    if verbose:
        print(" ".join(cmd), flush=True)
    started = time.time()
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        sys.stderr.write(res.stdout + res.stderr)
        raise RuntimeError("nvcc failed building libbicadmm.so")
    os.replace(tmp, LIB)
    # Stamp the library with the time the compiler started, so a source edited while it ran
    # is seen as newer than the library and triggers the next build.
    os.utime(LIB, (started, started))
    return LIB


if __name__ == "__main__":
    force = "--force" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas-v" in sys.argv else []
    print(build(force=force or bool(extra), verbose=True, extra=extra))

"""Build the in-tree CUDA library ``libptycho.so`` for B300 (sm_103a).

    python -m paper_2202_03144_b300.build [--force]

nvcc cross-compiles without a GPU.  Every ``csrc/*.cu`` translation unit is
compiled in parallel into ``_build/`` and the objects are linked into the
library.  It is rebuilt only when a source under ``csrc/`` or ``include/`` is
newer than the shared object.
"""
from __future__ import annotations

import concurrent.futures
import glob
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libptycho.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]
OBJDIR = os.path.join(PKG, "_build")


def _sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))
                  + glob.glob(os.path.join(ROOT, "include", "*.h")))


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in _sources())


def _compile(nvcc: str, src: str, obj: str, extra: list[str], verbose: bool):
    cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", "-o", obj, src]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    return subprocess.run(cmd, capture_output=True, text=True)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit under csrc/ in parallel, then link."""
    if not force and not stale():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    extra = os.environ.get("PTYCHO_NVCC_EXTRA", "").split()  # e.g. tuning macros
    units = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    os.makedirs(OBJDIR, exist_ok=True)
    objs = [os.path.join(OBJDIR, os.path.basename(u)[:-3] + ".o") for u in units]
    jobs = min(len(units), os.cpu_count() or 1)
    with concurrent.futures.ThreadPoolExecutor(max_workers=jobs) as ex:
        results = list(ex.map(lambda uo: _compile(nvcc, uo[0], uo[1], extra, verbose), zip(units, objs)))
    for u, res in zip(units, results):
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed on {os.path.basename(u)} ({res.returncode}):\n{res.stderr[-4000:]}")
        if verbose:
            sys.stderr.write(res.stderr)
    link = [nvcc, *ARCH, "-shared", "-o", LIB + ".tmp", *objs]
    res = subprocess.run(link, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed ({res.returncode}):\n{res.stderr[-4000:]}")
    os.replace(LIB + ".tmp", LIB)
    for o in objs:  # every build is a full one: keep only the library
        os.remove(o)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))

"""In-tree build of libswe.so for sm_103a (nvcc, no cmake).

Translation units compile in parallel into ``_build/`` and link into
``paper_2301_12010_gb300/libswe.so``; both are git-ignored.  The checked
build (``build(checked=True)``: every device index compared with its extent
before the access, SWE_CHECKED) goes to ``_build_checked/`` and
``libswe_checked.so``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import sys
from typing import List, Tuple

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libswe.so")
OUT_DIR_CHECKED = os.path.join(ROOT, "_build_checked")
LIB_CHECKED = os.path.join(PKG, "libswe_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + os.path.join(ROOT, "include")]



def _shapes() -> Tuple[int, ...]:
    """Indices of the tile shapes declared in the SWE_SHAPES table of swe_launch.h."""
    with open(os.path.join(CSRC, "swe_launch.h")) as f:
        text = f.read()
    table = text[text.index("#define SWE_SHAPES(X)"):]
    table = table[:table.index("\n\n")]
    return tuple(int(k) for k in re.findall(r"\bX\((\d+),", table))


# (source, extra flags, object name): one unit per (precision, tile shape) for
# the stage kernels and one per shape for the batch kernel, compiled in parallel
SHAPES = _shapes()
UNITS: List[Tuple[str, List[str], str]] = (
    [("swe_kernels.cu", ["-DSWE_PREC=%d" % p, "-DSWE_SHAPE=%d" % k], "swe_kernels_f%d_s%d.o" % (p, k))
     for p in (32, 64) for k in SHAPES]
    + [("swe_batch_kernels.cu", ["-DSWE_SHAPE=%d" % k], "swe_batch_kernels_s%d.o" % k) for k in SHAPES]
    + [("swe_shapes.cu", [], "swe_shapes.o"), ("swe_api.cu", [], "swe_api.o"), ("swe_aux.cu", [], "swe_aux.o"),
       ("swe_noalloc.cu", [], "swe_noalloc.o"), ("swe_batch.cu", [], "swe_batch.o"),
       ("swe_multi.cu", [], "swe_multi.o"), ("swe_fused.cu", [], "swe_fused.o"),
       ("swe_shore.cu", [], "swe_shore.o"), ("swe_batch64_kernels.cu", [], "swe_batch64_kernels.o"),
       ("swe_batch_shore.cu", [], "swe_batch_shore.o"),
       ("swe_autotune.cu", [], "swe_autotune.o")]
)


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libswe.so")


def _sources() -> List[str]:
    out = [os.path.abspath(__file__)]
    for d in (CSRC, os.path.join(ROOT, "include")):
        for f in os.listdir(d):
            if f.endswith((".cu", ".cuh", ".h")):
                out.append(os.path.join(d, f))
    return out


def up_to_date(checked: bool = False) -> bool:
    lib = LIB_CHECKED if checked else LIB
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False, extra: List[str] | None = None, checked: bool = False) -> str:
    lib = LIB_CHECKED if checked else LIB
    out_dir = OUT_DIR_CHECKED if checked else OUT_DIR
    if not force and up_to_date(checked):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    cc = nvcc()
    extra = list(extra or []) + (["-DSWE_CHECKED"] if checked else [])

    def compile_unit(u):
        src, fl, obj = u
        cmd = [cc] + ARCH + FLAGS + fl + extra + ["-c", os.path.join(CSRC, src), "-o", os.path.join(out_dir, obj)]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        return r.stdout + r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(len(UNITS), max(2, os.cpu_count() or 2))) as ex:
        logs = list(ex.map(compile_unit, UNITS))
    if verbose:
        for l in logs:
            sys.stderr.write(l)
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [cc] + ARCH + ["-shared", "-o", tmp] + [os.path.join(out_dir, u[2]) for u in UNITS]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))

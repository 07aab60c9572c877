"""Build the CUDA library libsc.so in-tree with nvcc (sm_103a only).

Each .cu translation unit compiles in parallel to an object under _build/,
then nvcc links them into paper_2106_15789_gb300/libsc.so. No CMake, no torch
extension machinery: the library exposes a plain C ABI (include/sc.h).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libsc.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["sc_api.cu", "sc_smooth.cu", "sc_smooth_tile.cu", "sc_smooth_ws.cu", "sc_smooth_fir.cu", "sc_smooth_ws16.cu", "sc_smooth_z.cu", "sc_smooth_p.cu", "sc_noise.cu", "sc_noise_scale.cu", "sc_linker.cu", "sc_flagger.cu", "sc_static.cu",
           "sc_gauss.cu"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsc.so")


def _flags(extra=()):
    # every compiler warning is an error (a value-less return in a bool
    # function, for one, is undefined behaviour the optimiser may exploit)
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Werror", "all-warnings", "-Xcompiler", "-fPIC", "-I",
                   os.path.join(ROOT, "include"), "-I", CSRC, *extra]


def _compile(src: str, verbose: bool, extra) -> str:
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj] + _flags(extra)
    if verbose:
        cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    return obj


def build(verbose: bool = False, extra=()) -> str:
    """Compile and link libsc.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, extra), SOURCES))
    tmp = LIB + ".tmp"
    cmd = [nvcc(), "-shared", "-o", tmp, *objs] + ARCH + ["-Xcompiler", "-fPIC"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))

"""Build libdfr.so in place: every CUDA / C++ source compiled for sm_103a in parallel, then
linked into one shared library beside this file (git-ignored). Run ``python -m
paper_2505_03932_gb300.build`` or call ``build()``."""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libdfr.so")
OBJ = os.path.join(HERE, "_build")
SOURCES = ["dfr_fwd_single_t16.cu", "dfr_fwd_single_sw_t16.cu", "dfr_fwd_batch_t16.cu",
           "dfr_fwd_batch_sw_t16.cu", "dfr_fwd_single_t32.cu", "dfr_fwd_single_sw_t32.cu",
           "dfr_fwd_batch_t32.cu", "dfr_fwd_batch_sw_t32.cu", "dfr_fwd_single_t8.cu",
           "dfr_fwd_single_sw_t8.cu", "dfr_fwd_batch_t8.cu", "dfr_fwd_batch_sw_t8.cu",
           "dfr_fwd.cu", "dfr_bwd.cu", "dfr_bwd_tile.cu", "dfr_coadd.cu", "dfr_bspline.cu",
           "dfr_host.cpp", "dfr_static.cu", "dfr_peaks.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdfr")


def _compile(src: str) -> str:
    obj = os.path.join(OBJ, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-I", os.path.join(ROOT, "include"), "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
    return obj


def build(verbose: bool = False) -> str:
    os.makedirs(OBJ, exist_ok=True)
    srcs = [s for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(_compile, srcs))
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "shared", "-o", LIB + ".tmp", *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(LIB + ".tmp", LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(verbose="-q" not in sys.argv)

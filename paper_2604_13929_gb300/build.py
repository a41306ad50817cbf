"""Build libspmc.so and libspnn.so in-tree with nvcc for sm_103a.

The translation units of both libraries are compiled in parallel and linked
into ``paper_2604_13929_gb300/_lib/`` (static CUDA runtime, so the libraries
need only the NVIDIA kernel-mode driver's libcuda at run time):

* libspmc -- the voxel Monte Carlo transport (include/spmc.h);
* libspnn -- the fluence surrogate's tensor-core kernels (include/spnn.h).

Usage::

    python -m paper_2604_13929_gb300.build [--verbose]
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
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libspmc.so")
NN_LIB = os.path.join(LIBDIR, "libspnn.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
SOURCES = ["spmc_api.cu", "spmc_transport_f32.cu", "spmc_transport_f64.cu", "spmc_probe.cu"]
NN_SOURCES = ["spnn_api.cu", "spnn_gemm.cu"]
TARGETS = {LIB: (SOURCES, "spmc"), NN_LIB: (NN_SOURCES, "spnn")}
# The FP64 transport evaluates the plain-definition formulas in their written
# order; contraction into fused multiply-adds would change its rounding.
PER_SOURCE_FLAGS = {"spmc_transport_f64.cu": ["-fmad=false"]}


def nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _flags(verbose: bool):
    f = ["-O3", "-std=c++17", ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-O2",
         f"-I{INCLUDE}", f"-I{CSRC}", "--expt-relaxed-constexpr"]
    if verbose:
        f += ["-Xptxas", "-v"]
    return f


def _deps(prefix):
    return ([os.path.join(CSRC, n) for n in os.listdir(CSRC) if n.startswith(prefix)]
            + [os.path.join(INCLUDE, prefix + ".h")])


def up_to_date() -> bool:
    for lib, (_, prefix) in TARGETS.items():
        if not os.path.exists(lib):
            return False
        t = os.path.getmtime(lib)
        if not all(os.path.getmtime(d) <= t for d in _deps(prefix)):
            return False
    return True


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(os.path.join(LIBDIR, "obj"), exist_ok=True)
    cc = nvcc()

    def compile_one(src):
        obj = os.path.join(LIBDIR, "obj", src.replace(".cu", ".o"))
        extra = PER_SOURCE_FLAGS.get(src, [])
        cmd = [cc, *_flags(verbose), *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stdout + r.stderr

    every = [src for srcs, _ in TARGETS.values() for src in srcs]
    with cf.ThreadPoolExecutor(len(every)) as ex:
        results = dict(zip(every, ex.map(compile_one, every)))
    if verbose:
        for _, log in results.values():
            sys.stderr.write(log)
    for lib, (srcs, _) in TARGETS.items():
        tmp = lib + f".{os.getpid()}.tmp"
        cmd = [cc, ARCH, "-shared", "-o", tmp, *[results[s][0] for s in srcs]]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose="--verbose" in sys.argv))

"""Build libpe3d.so in-tree with nvcc for sm_103a (no CMake, no torch extension).

Each translation unit compiles in parallel; the shared object links the CUDA
runtime statically.  `python -m paper_1711_00005_gb300.build` rebuilds it.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpe3d.so")
SOURCES = ["pe3d_api.cu", "pe3d_f32.cu", "pe3d_f64.cu", "pe3d_server.cu", "pe3d_static.cu",
           "pe3d_batch_f32.cu", "pe3d_batch_f64.cu", "pe3d_synth.cu", "pe3d_resident.cu",
           "pe3d_taylor_f32.cu", "pe3d_taylor_f64.cu"]
# the measured roofline denominators (L2 copy, FMA rates): a separate library
# that only the benchmark loads
PEAKS_LIB = os.path.join(HERE, "libpe3d_peaks.so")
PEAKS_SOURCE = "pe3d_peaks.cu"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Host code is compiled without floating-point contraction: the range at which
# a step evaluates the medium, r0 + (j+1) dr, decides which slice is active, and
# it must round as written (product, then sum) on every host, like the oracle;
# aarch64 compilers otherwise fuse it into one FMA and can pick the other slice
# when r* falls on a slice boundary.
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2,-ffp-contract=off", "--expt-relaxed-constexpr",
              "-Xptxas", "-v", "-I", os.path.join(HERE, "..", "include")]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(PEAKS_LIB):
        return True
    t = min(os.path.getmtime(LIB), os.path.getmtime(PEAKS_LIB))
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "pe3d.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()

    def compile_one(src: str):
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *NVCC_FLAGS, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        with open(os.path.join(BUILD, src + ".log"), "w") as f:
            f.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stderr[-4000:]}")
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES) + 1) as ex:
        objs = list(ex.map(compile_one, SOURCES + [PEAKS_SOURCE]))
    peaks_obj = objs.pop()
    tmp = PEAKS_LIB + ".tmp"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, peaks_obj, "-cudart", "static", "-lpthread", "-ldl",
                        "-lrt"], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link of {os.path.basename(PEAKS_LIB)} failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, PEAKS_LIB)
    tmp = LIB + ".tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static", "-lpthread", "-ldl", "-lrt"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)

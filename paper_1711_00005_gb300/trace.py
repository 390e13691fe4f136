"""Sub-step tracing of the range march (one GPU).

Builds a copy of the library with -DPE3D_TRACE into _build/trace/ and marches
the walled 100 Hz grid for a few steps.  The trace build makes thread 0 of
every CTA record clock64() at each sub-step of the two phases and around the
grid barriers.  Prints the median and maximum SM cycles of each sub-step over
the CTAs:

    python -m paper_1711_00005_gb300.trace [--steps 20] [--exec 3]

The traced library is separate from libpe3d.so and is never loaded by the
library's users.
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import ctypes
import os
import subprocess
import sys

import numpy as np

from . import build as _build

TRACE_DIR = os.path.join(_build.BUILD, "trace")
TRACE_LIB = os.path.join(TRACE_DIR, "libpe3d_trace.so")
SLOTS = 24
NAMES_A = ["tma_wait", "F1", "scan1", "F2+B1", "scan2", "B2+sync", "store"]
NAMES_B = ["tma_wait", "F1", "scan1", "F2+B1", "scan2", "B2+sync", "epilogue"]


def build_traced() -> str:
    os.makedirs(TRACE_DIR, exist_ok=True)
    cc = _build.nvcc()
    flags = [f for f in _build.NVCC_FLAGS if f not in ("-Xptxas", "-v")]

    def one(src):
        obj = os.path.join(TRACE_DIR, src.replace(".cu", ".o"))
        subprocess.run([cc, *_build.ARCH, *flags, "-DPE3D_TRACE", "-c", os.path.join(_build.CSRC, src), "-o", obj],
                       check=True, capture_output=True)
        return obj

    with cf.ThreadPoolExecutor(len(_build.SOURCES)) as ex:
        objs = list(ex.map(one, _build.SOURCES))
    subprocess.run([cc, *_build.ARCH, "-shared", "-o", TRACE_LIB, *objs, "-cudart", "static", "-lpthread", "-ldl",
                    "-lrt"], check=True, capture_output=True)
    return TRACE_LIB


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--exec", type=int, default=3, help="1 stream, 3 persistent")
    a = ap.parse_args(argv)
    import torch

    import paper_1711_00005_gb300 as P
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import workloads

    L = P.load_library(build_traced())
    L.pe3d_trace_read.argtypes = [ctypes.c_void_p, ctypes.c_size_t]
    wl = workloads.config2(steps=a.steps)
    g = wl.grid
    plan = P.Plan.for_grid(g, fp32=True, exec_mode=a.exec)
    plan.set_medium(torch.from_numpy(wl.n2).cuda(), wl.slice_r)
    u0 = torch.from_numpy(wl.u0.astype(np.complex64)).cuda()
    plan.march(u0, g.r0, g.steps, g.steps)
    torch.cuda.synchronize()
    buf = np.zeros((4096, SLOTS), np.int64)
    L.pe3d_trace_read(buf.ctypes.data, buf.nbytes)
    inf = plan.info()
    ng = 256 // inf["zthreads"]
    nA = (g.Ntheta + ng - 1) // ng
    nB = (g.Nz + inf["ttile"] - 1) // inf["ttile"]
    A, B = buf[:nA, 0:8], buf[:nB, 8:16]
    dA, dB = np.diff(A, axis=1), np.diff(B, axis=1)
    print("layout", {k: inf[k] for k in ("ldz", "zthreads", "zchunk", "ttile", "tchunk", "grid")})
    print("depth phase (cycles, median/max):",
          {n: (int(np.median(dA[:, i])), int(dA[:, i].max())) for i, n in enumerate(NAMES_A)})
    print("azimuth phase (cycles, median/max):",
          {n: (int(np.median(dB[:, i])), int(dB[:, i].max())) for i, n in enumerate(NAMES_B)})
    if a.exec == 3:
        G = inf["grid"]
        Bb = buf[:G, 16:20]
        print("grid barriers (cycles, median/max): after depth phase", int(np.median(Bb[:, 1] - Bb[:, 0])),
              int((Bb[:, 1] - Bb[:, 0]).max()), "; after azimuth phase", int(np.median(Bb[:, 3] - Bb[:, 2])),
              int((Bb[:, 3] - Bb[:, 2]).max()))
    plan.close()


if __name__ == "__main__":
    main()

"""Sub-step tracing of the range march (one GPU).

Builds a copy of the library with -DPE3D_TRACE into _build/trace/ and marches
one workload for a few steps.  In the trace build, thread 0 of every CTA adds
the SM cycles since its previous mark to the slot of the interval that ends
there, over every unit and range step.  Prints, per interval, the mean over
the CTAs of the cycles spent per range step (their sum is the step time):

    python -m paper_1711_00005_gb300.trace [--workload medium-100Hz] [--steps 20] [--exec 3]

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
# interval ending at each mark (slot number -> name)
NAMES = {
    0: "A: before unit", 1: "A: TMA wait", 2: "A: F1", 3: "A: scan1", 4: "A: F2+B1", 5: "A: scan2",
    6: "A: B2+sync", 7: "A: store v", 16: "A: after units", 17: "barrier 1",
    8: "B: before tile", 9: "B: TMA wait", 10: "B: F1", 11: "B: scan1", 12: "B: F2+B1", 13: "B: scan2",
    14: "B: B2+SM+sync", 15: "B: epilogue", 18: "B: after tiles", 19: "barrier 2",
}
# the resident march (exec 4)
NAMES_RESIDENT = {
    20: "step start (coefficient copies)", 0: "slice change", 1: "A: zero-carry solve + publish",
    2: "A: exchange + sweep", 3: "A: sync", 4: "A: carried solve + v", 5: "coefficients wait + sync",
    6: "B: zero-carry solve + publish", 7: "B: exchange + sweep", 8: "B: sync", 9: "B: carried solve + u",
    10: "B: sync", 11: "B: stencil + snapshot", 12: "B: w + syncs",
}


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
    ap.add_argument("--workload", choices=["medium-100Hz", "periodic-200Hz", "batched-25-400Hz", "served-mix"],
                    default="medium-100Hz")
    ap.add_argument("--members", type=int, default=32, help="batched: the highest-frequency members only")
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--exec", type=int, default=3, help="1 stream, 3 persistent, 4 resident")
    ap.add_argument("--autotune-steps", type=int, default=100, help="choose the layout as bench.py does (0: off)")
    a = ap.parse_args(argv)
    import torch

    import paper_1711_00005_gb300 as P
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import workloads

    L = P.load_library(build_traced())
    L.pe3d_trace_read.argtypes = [ctypes.c_void_p, ctypes.c_size_t]
    L.pe3d_trace_read_resident.argtypes = [ctypes.c_void_p, ctypes.c_size_t]
    read = L.pe3d_trace_read_resident if a.exec == 4 else L.pe3d_trace_read
    if a.workload in ("batched-25-400Hz", "served-mix"):
        return trace_batched(P, L, workloads, a)
    make = workloads.config2 if a.workload == "medium-100Hz" else workloads.config3
    wl = make(steps=a.steps)
    g = wl.grid
    plan = P.Plan.for_grid(g, fp32=True, exec_mode=a.exec)
    plan.set_medium(torch.from_numpy(wl.n2).cuda(), wl.slice_r)
    if a.autotune_steps > 0:
        P.pe3d_autotune(plan.h, g.r0, min(a.autotune_steps, g.steps))
    u0 = torch.from_numpy(wl.u0.astype(np.complex64)).cuda()
    buf = np.zeros((4096, SLOTS), np.int64)
    plan.march(u0, g.r0, g.steps, g.steps)          # warm-up, then clear the counters
    read(buf.ctypes.data, buf.nbytes)
    plan.march(u0, g.r0, g.steps, g.steps)
    read(buf.ctypes.data, buf.nbytes)
    inf = plan.info()
    G = inf["grid"] if a.exec in (3, 4) else 4096
    rows = buf[:G]
    rows = rows[rows.sum(axis=1) != 0]
    print("workload", g.name, "layout", {k: inf[k] for k in ("ldz", "zthreads", "zchunk", "ttile", "tchunk", "grid")})
    report(rows, g.steps, NAMES_RESIDENT if a.exec == 4 else NAMES)
    plan.close()


def report(rows, steps, names=NAMES):
    print(f"{'interval':18s} {'mean':>8s} {'max':>8s}   (SM cycles per range step, over {len(rows)} CTAs)")
    tot = 0.0
    for s_, name in names.items():
        v = rows[:, s_] / steps
        tot += v.mean()
        print(f"{name:18s} {v.mean():8.0f} {v.max():8.0f}")
    print(f"{'step total':18s} {tot:8.0f}")


def trace_batched(P, L, workloads, a):
    """The batched launch of the highest-frequency members of the 32-frequency
    batch, or of the first requests of the served stream, all marched a.steps
    steps."""
    import torch
    if a.workload == "served-mix":
        reqs = workloads.config5_stream(rate=200.0, duration=3.0, seed=5)[:a.members]
        grids = [workloads.config5_grid(r, max_steps=a.steps) for r in reqs]
        wls = [workloads.config5_member(r, g, n_slices=1) for r, g in zip(reqs, grids)]
    else:
        grids = workloads.config4_grids()[-a.members:]
        for g in grids:
            g.steps = a.steps
        wls = [workloads.config4_member(g) for g in grids]
    for g in grids:
        g.stride = g.steps
    stream = torch.cuda.Stream()
    plans, u0s, outs = [], [], []
    for wl in wls:
        g = wl.grid
        h = P.pe3d_plan(g.Nz, g.Ntheta, g.dz, g.dtheta, g.dr, g.k0,
                        P.PE3D_PERIODIC if g.periodic else P.PE3D_WALLED, P.PE3D_FP32, stream)
        P.pe3d_set_medium(h, torch.from_numpy(wl.n2).cuda(), wl.slice_r)
        plans.append(h)
        u0s.append(torch.from_numpy(wl.u0.astype(np.complex64)).cuda())
        outs.append(torch.empty((1, g.Ntheta, g.Nz), dtype=torch.complex64, device="cuda"))
    buf = np.zeros((4096, SLOTS), np.int64)
    L.pe3d_trace_read_batched.argtypes = [ctypes.c_void_p, ctypes.c_size_t]
    for _ in range(2):    # warm-up, then the traced launch
        L.pe3d_trace_read_batched(buf.ctypes.data, buf.nbytes)
        P.pe3d_march_batched(plans, u0s, [g.r0 for g in grids], [g.steps for g in grids],
                             [g.stride for g in grids], outs)
    L.pe3d_trace_read_batched(buf.ctypes.data, buf.nbytes)
    inf = P.pe3d_plan_info(plans[0])
    print("workload", a.workload, len(grids), "members", [(g.Nz, g.Ntheta) for g in grids[:4]], "...",
          "grid", inf["grid"])
    rows = buf[:inf["grid"]]
    report(rows[rows.sum(axis=1) != 0], a.steps)
    for h in plans:
        P.pe3d_destroy(h)


if __name__ == "__main__":
    main()

#!/usr/bin/env python3
"""Benchmark of the 3D wide-angle PE range march on GB300.

One bench step = one pass of the whole hot path over the medium-sized
100 Hz workload (Nz=1067 x Ntheta=256, 2000 range steps, 101 medium slices):
FP64 coefficient setup of every slice's depth systems (pe3d_set_medium from a
device-resident n^2), then the march itself (per-step FP64 azimuth setup,
then the complex-FP32 range steps in one persistent cooperative launch, in
the layout the autotuner picks), all through the library's C ABI.  The
metric is grid-point range-steps per second, at a relative L2 error against
the FP64 oracle that the run measures and reports.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (torchrun) runs N independent replicas (one march per GPU, no
collective on the data path) and reports the whole-job rate.
`--impl reference` times the FP64 CPU oracle on this machine's cores on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

os.environ.setdefault("OMP_WAIT_POLICY", "PASSIVE")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads  # noqa: E402

METRIC = "grid-point range-steps/s at ≤1e-4 rel-L2 vs FP64 oracle; p50/p99 solve latency"
UNIT = "grid-point range-steps/s"
BYTES_PER_POINT_STEP = {"fp32": 40, "fp64": 80}
FALLBACK_HBM_GBS = 6800.0
# FP64 marches are bound by GB300's FP64 pipe: ~80 real flops per grid-point
# range-step (theta and depth stencils of the RHS, the two elimination sweeps)
FLOPS_PER_POINT_STEP = 80
NOMINAL_FP64_GFLOPS = 1250.0
# per-step depth set-up of an interpolated medium, per grid point and range
# step: n^2 = (1-t) a + t b (6), d/e + mu = ae n^2 + ce + mu (10), |den|^2 (3),
# the reciprocal (1) and mu = -conj(den) / |den|^2 (2) -- 22 real FP64 flops
SETUP_FLOPS_PER_POINT_STEP = 22


# ---------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------

def rank_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def init_dist(backend: str):
    import torch.distributed as dist
    if int(os.environ.get("WORLD_SIZE", 1)) > 1 and not dist.is_initialized():
        dist.init_process_group(backend=backend)
    return dist


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def reduce_max(x: float, device=None) -> float:
    """Max over ranks (identity on one process)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def live_peaks():
    """L2 copy bandwidth and FMA rates measured on this GPU now (before the
    timed region), by the probes of paper_1711_00005_gb300.peaks."""
    from paper_1711_00005_gb300 import peaks
    try:
        return peaks.measure()
    except Exception as e:          # reported, not fatal: the HBM roofline stands alone
        return {"error": str(e)}


def l2_roofline(achieved_gbs, lp):
    if not lp or "l2_gbs" not in lp:
        return None
    return {"bound": "l2", "achieved": achieved_gbs, "peak": lp["l2_gbs"], "unit": "GB/s",
            "frac": achieved_gbs / lp["l2_gbs"],
            "peak_source": "measured in this run: L2-resident read+write copy (pe3d_peak_l2_copy), "
                           + ", ".join(f"{k} {v:.0f} GB/s" for k, v in lp["l2_by_footprint_gbs"].items())}


def fp64_peak(lp):
    """(TFLOP/s, source) of the FP64 pipe: measured in this run, else nominal."""
    if lp and lp.get("fp64_tflops"):
        return lp["fp64_tflops"], "measured in this run (pe3d_peak_fma, FP64 FMA chains)"
    return NOMINAL_FP64_GFLOPS / 1e3, "nominal FP64 rate of the profiling recipe"


def oracle_one_thread(wl, steps, interp=False, taylor=False):
    """The oracle at one thread on a bounded sample: the first `steps` range
    steps of the workload."""
    _, dt = oracle_run(wl, steps, 1, interp, taylor)
    return {"value": wl.grid.points * steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {steps} range steps of {wl.grid.name}, one thread ({dt:.1f} s)"}


# the files the range-march kernels are built from
MARCH_SOURCES = ("pe3d_device.cuh", "pe3d_f32.cu", "pe3d_f64.cu", "pe3d_kernels.cuh", "pe3d_march_impl.cuh",
                 "pe3d_resident.cuh", "pe3d_resident.cu")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1711_00005_gb300", "csrc")
    for name in MARCH_SOURCES:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if the kernel
    sources are unchanged since it was taken (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        e = d[kernel][workload]
        if e.get("source_sha256") != kernel_source_hash():
            return None
        return float(e["dram_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.proc = None
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
            if gpu_id:
                cmd += ["-i", gpu_id]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def gpu_uuid():
    try:
        import torch
        u = torch.cuda.get_device_properties(torch.cuda.current_device()).uuid
        s = str(u)
        return s if s.startswith("GPU-") else "GPU-" + s
    except Exception:
        return None


def relerr_series(got, ref):
    return [float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())) for a, b in zip(got, ref)]


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

WORKLOADS = {
    "medium-100Hz": ("fp32", lambda: workloads.config2()),
    "medium-100Hz-fp64": ("fp64", lambda: workloads.config2()),
    "walled-50Hz": ("fp64", lambda: workloads.config1()),
    "periodic-200Hz": ("fp32", lambda: workloads.config3()),
    "medium-100Hz-interp": ("fp32", lambda: workloads.config2()),
    "medium-100Hz-taylor": ("fp32", lambda: workloads.config2()),
}
# workloads marched with the Taylor form of Eq. 3
TAYLOR_WORKLOADS = {"medium-100Hz-taylor"}
# workloads whose n^2 is interpolated linearly in range, with the FP64 depth
# systems set up for every range step
INTERP_WORKLOADS = {"medium-100Hz-interp"}


def oracle_run(wl, steps: int, nthreads: int, interp: bool = False, taylor: bool = False):
    import oracle
    L = oracle.load()
    g = wl.grid
    stride = g.stride if steps % g.stride == 0 else steps
    t = time.perf_counter()
    out = L.march(g, wl.n2, wl.slice_r, wl.u0, steps=steps, stride=stride, nthreads=nthreads, interp=interp,
                  taylor=taylor)
    return out, time.perf_counter() - t


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------

def run_reference(args):
    rank, world, _ = rank_info()
    if world > 1:
        init_dist("gloo")
        if rank != 0:
            barrier()
            return 0
    if args.workload not in WORKLOADS:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm covers the single-march workloads; "
                          f"{args.workload} reports its oracle sample as cpu_baseline in its own line"}), flush=True)
        if world > 1:
            barrier()
        return 0
    import oracle
    precision, make = WORKLOADS[args.workload]
    wl = make()
    g = wl.grid
    cores = oracle.default_threads()
    sample_steps = min(g.steps, args.ref_sample_steps)
    interp = args.workload in INTERP_WORKLOADS
    taylor = args.workload in TAYLOR_WORKLOADS
    for _ in range(args.warmup):
        oracle_run(wl, sample_steps, cores, interp, taylor)
    times = []
    for _ in range(args.steps):
        _, dt = oracle_run(wl, sample_steps, cores, interp, taylor)
        times.append(dt)
    per = statistics.mean(times)
    value = g.points * sample_steps / per
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": g.name + ("-interp" if interp else "") + ("-taylor" if taylor else ""),
                   "sample_range_steps": sample_steps,
                   "Nz": g.Nz, "Ntheta": g.Ntheta},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"first {sample_steps} of {g.steps} range steps of {g.name}, "
                                   f"FP64 C oracle, OpenMP over systems"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        barrier()
    return 0


def run_ours(args):
    import torch
    rank, world, local = rank_info()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    init_dist("nccl")
    from paper_1711_00005_gb300 import build
    if rank == 0 or world == 1:
        build.build()
    barrier()
    import paper_1711_00005_gb300 as P

    precision, make = WORKLOADS[args.workload]
    fp32 = precision == "fp32"
    interp = args.workload in INTERP_WORKLOADS
    taylor = args.workload in TAYLOR_WORKLOADS
    wl = make()
    g = wl.grid
    if interp:
        g.name += "-interp"
    if taylor:
        g.name += "-taylor"
    if args.range_steps:                      # a truncated march (profiling cases)
        g.steps = min(g.steps, args.range_steps)
        g.stride = max(1, min(g.stride, g.steps))
    point_steps = g.point_steps
    cdt = np.complex64 if fp32 else np.complex128
    tcdt = torch.complex64 if fp32 else torch.complex128

    # CPU baseline + oracle reference (rank 0, before any GPU work is timed)
    cpu = None
    ref = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        cores = oracle.default_threads()
        ref, dt = oracle_run(wl, g.steps, cores, interp, taylor)
        cpu = {"value": g.points * g.steps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"the full {g.steps}-step march of {g.name} (FP64 C oracle, OpenMP over "
                         f"systems, {dt:.1f} s)",
               "one_thread": oracle_one_thread(wl, min(g.steps, args.one_thread_steps), interp, taylor)}
    lp = live_peaks() if rank == 0 else None

    stream = torch.cuda.Stream(device=dev)
    n2_dev = torch.from_numpy(wl.n2).to(dev)
    u0_dev = torch.from_numpy(wl.u0.astype(cdt)).to(dev)
    out_mode = {"field": 0, "pressure": 1, "tl": 2}[args.output]
    odt = tcdt if out_mode != 2 else (torch.float32 if fp32 else torch.float64)
    out_dev = torch.empty((g.n_out, g.Ntheta, g.Nz), dtype=odt, device=dev)
    torch.cuda.synchronize()
    plan = P.pe3d_plan(g.Nz, g.Ntheta, g.dz, g.dtheta, g.dr, g.k0,
                       P.PE3D_PERIODIC if g.periodic else P.PE3D_WALLED,
                       P.PE3D_FP32 if fp32 else P.PE3D_FP64, stream)
    exec_mode = args.exec
    if taylor:
        P.pe3d_set_option(plan, P.PE3D_OPT_SCHEME, P.PE3D_SCHEME_TAYLOR)
    P.pe3d_set_option(plan, P.PE3D_OPT_EXEC, exec_mode)
    P.pe3d_set_option(plan, P.PE3D_OPT_TIMING, 1)
    P.pe3d_set_option(plan, P.PE3D_OPT_OUTPUT, out_mode)
    if args.rc:
        P.pe3d_set_option(plan, P.PE3D_OPT_RC_EVERY, args.rc)
    if interp:
        P.pe3d_set_option(plan, P.PE3D_OPT_MEDIUM_INTERP, 1)

    def step():
        P.pe3d_set_medium(plan, n2_dev, wl.slice_r)
        P.pe3d_march(plan, u0_dev, g.r0, g.steps, g.stride, out_dev)

    if args.autotune_steps > 0:   # choose the layout by timing candidates (untimed set-up)
        P.pe3d_set_medium(plan, n2_dev, wl.slice_r)
        P.pe3d_autotune(plan, g.r0, min(args.autotune_steps, g.steps))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # parity of this run's output against the oracle (pressure and transmission
    # loss through |p| = 10^(-TL/20), as in the tests)
    err = None
    if ref is not None:
        got = out_dev.cpu().numpy()
        if out_mode == 0:
            err = max(relerr_series(got, ref))
        else:
            import oracle
            p_ref = oracle.pressure(ref, oracle.snapshot_ranges(g.r0, g.dr, g.steps, g.stride), g.k0)
            if out_mode == 1:
                err = max(relerr_series(got, p_ref))
            else:
                err = max(relerr_series(10.0 ** (-got.astype(np.float64) / 20.0), np.abs(p_ref)))

    # timed region: K steps, CUDA events on the plan's stream
    launches0 = P.pe3d_plan_info(plan)["total_launches"]
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(gpu_uuid())
    kernel_ns, setup_ns = [], []
    barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
        inf = P.pe3d_plan_info(plan)
        kernel_ns.append(inf["kernel_ns"])
        setup_ns.append(inf["setup_ns"])
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    info = P.pe3d_plan_info(plan)
    launches = info["total_launches"] - launches0
    t_local = ev0.elapsed_time(ev1) / 1e3
    t = reduce_max(t_local, dev)
    total_units = reduce_sum(point_steps * args.steps, dev)

    # end to end: host (pinned) buffers through the same C ABI calls, copies timed
    n2_h = torch.from_numpy(wl.n2).pin_memory()
    u0_h = torch.from_numpy(wl.u0.astype(cdt)).pin_memory()
    out_h = torch.empty((g.n_out, g.Ntheta, g.Nz), dtype=odt).pin_memory()
    e2e_steps = max(1, min(args.steps, 5))
    P.pe3d_set_medium(plan, n2_h, wl.slice_r)
    P.pe3d_march(plan, u0_h, g.r0, g.steps, g.stride, out_h)
    barrier()
    t_sm = t_m = 0.0
    e2e_each = []
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        ta = time.perf_counter()
        P.pe3d_set_medium(plan, n2_h, wl.slice_r)
        tb = time.perf_counter()
        P.pe3d_march(plan, u0_h, g.r0, g.steps, g.stride, out_h)
        tc = time.perf_counter()
        t_sm += tb - ta
        t_m += tc - tb
        e2e_each.append(tc - ta)
    t_e2e = reduce_max((time.perf_counter() - t0) / e2e_steps, dev)

    # plain FP64 GPU march of the same workload, for comparison
    fp64_value = None
    if fp32 and not args.no_fp64_compare and not interp and not taylor:
        u064 = torch.from_numpy(wl.u0).to(dev)
        o64 = torch.empty((g.n_out, g.Ntheta, g.Nz), dtype=torch.complex128, device=dev)
        p64 = P.pe3d_plan(g.Nz, g.Ntheta, g.dz, g.dtheta, g.dr, g.k0,
                          P.PE3D_PERIODIC if g.periodic else P.PE3D_WALLED, P.PE3D_FP64, stream)
        P.pe3d_set_medium(p64, n2_dev, wl.slice_r)
        P.pe3d_march(p64, u064, g.r0, g.steps, g.stride, o64)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        reps = 3
        for _ in range(reps):
            P.pe3d_set_medium(p64, n2_dev, wl.slice_r)
            P.pe3d_march(p64, u064, g.r0, g.steps, g.stride, o64)
        e1.record(stream)
        torch.cuda.synchronize()
        fp64_value = point_steps * reps / (e0.elapsed_time(e1) / 1e3)
        if ref is not None:
            fp64_err = max(relerr_series(o64.cpu().numpy(), ref))
        else:
            fp64_err = None
        P.pe3d_destroy(p64)

    if rank == 0:
        peak, peak_kind = measured_peaks()
        kns = statistics.mean(kernel_ns) if kernel_ns and kernel_ns[0] > 0 else None
        bpp = BYTES_PER_POINT_STEP[precision]
        if taylor:      # the depth phase also reads the second factor's multipliers
            bpp += BYTES_PER_POINT_STEP[precision] // 5
        roof = None
        if kns and fp32:
            achieved = bpp * point_steps / (kns * 1e-9) / 1e9
            if taylor:
                kname = ("k_march_persistent<float2> (Taylor form)" if info["exec"] == 3
                         else "k_phaseA_taylor<float2> + k_phaseB<float2> (per-step launches)")
            else:
                kname = "k_march_resident<float2>" if info["exec"] == 4 else "k_march_persistent<float2>"

            roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    "peak_source": f"{peak_kind} hbm_gbs", "kernel": kname,
                    "algorithmic_bytes_per_launch": bpp * point_steps, "kernel_ms": kns / 1e6,
                    "traffic": recorded_traffic(kname, g.name),
                    # the field stays in L2: the same achieved bytes against the L2 copy rate
                    "l2": l2_roofline(achieved, lp)}
        elif kns:
            achieved = FLOPS_PER_POINT_STEP * point_steps / (kns * 1e-9) / 1e12
            kname = "k_march_persistent<double2>"
            p64, p64_src = fp64_peak(lp)
            roof = {"bound": "alu", "achieved": achieved, "peak": p64, "unit": "TFLOP/s",
                    "frac": achieved / p64, "peak_source": p64_src,
                    "kernel": kname, "algorithmic_flops_per_launch": FLOPS_PER_POINT_STEP * point_steps,
                    "kernel_ms": kns / 1e6, "traffic": recorded_traffic(kname, g.name),
                    "hbm": {"achieved": BYTES_PER_POINT_STEP[precision] * point_steps / (kns * 1e-9) / 1e9,
                            "peak": peak, "unit": "GB/s",
                            "frac": BYTES_PER_POINT_STEP[precision] * point_steps / (kns * 1e-9) / 1e9 / peak}}
        line = {
            "metric": METRIC,
            "value": total_units / t,
            "unit": UNIT,
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": t / args.steps * 1e3,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32" if fp32 else "f64",
            "data": "synthetic",
            "config": {
                "workload": g.name, "Nz": g.Nz, "Ntheta": g.Ntheta, "range_steps": g.steps,
                "medium_slices": len(wl.slice_r), "point_steps_per_march": point_steps,
                "precision": "complex64 march, FP64 coefficient setup" if fp32 else "complex128",
                "exec": ["auto", "stream", "graph", "persistent", "resident"][info["exec"]],
                "fp64_residual_correction_every": args.rc or None,
                "scheme": ("Taylor form of Eq. 3: [1 -+ (d/2)(X/2 - X^2/8)], two tridiagonal factors"
                           if taylor else "Eq. 4 (Pade)"),
                "medium": ("n^2 interpolated linearly in range between the slices; FP64 depth systems set up "
                           "for every range step" if interp else
                           "piecewise constant in range, FP64 depth systems set up per slice"),
                "output": {"field": "envelope u", "pressure": "p = u H0(k0 r)",
                           "tl": "-20 log10 |p| (dB)"}[args.output],
                "layout": {k: info[k] for k in ("ldz", "zthreads", "zchunk", "ttile", "tchunk", "grid")},
                "layout_by": "autotune" if args.autotune_steps > 0 else "default heuristic",
                "l2": "flushed each step: the step re-reads the 441 MB n^2 and rewrites 220 MB of "
                      "coefficients (> 129 MB L2) before the march",
                "parallelism": f"replicas x{world}",
            },
            "max_rel_l2_vs_oracle": err,
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": {"value": total_units / args.steps / t_e2e, "unit": UNIT,
                    "h2d_bytes_per_step": int(wl.n2.nbytes + wl.u0.astype(cdt).nbytes),
                    "d2h_bytes_per_step": int(out_h.numel() * out_h.element_size()),
                    "ms_per_step": t_e2e * 1e3,
                    "ms_min_median_max": [round(1e3 * min(e2e_each), 3), round(1e3 * statistics.median(e2e_each), 3),
                                          round(1e3 * max(e2e_each), 3)],
                    "set_medium_ms": t_sm / e2e_steps * 1e3, "march_ms": t_m / e2e_steps * 1e3},
            "gpu_launches": int(launches),
            "clocks": clocks,
        }
        sns = statistics.mean(setup_ns) if setup_ns and setup_ns[0] > 0 else None
        if sns:
            line["setup"] = {"ms": sns / 1e6,
                             "kernels": "k_setupA_lerp + k_setupB" if interp else "k_setupB",
                             "note": "per-march set-up inside pe3d_march, CUDA events on the plan's stream"}
            if interp:
                fl = SETUP_FLOPS_PER_POINT_STEP * point_steps
                p64, p64_src = fp64_peak(lp)
                line["setup"].update({"bound": "alu", "achieved": fl / (sns * 1e-9) / 1e12, "unit": "TFLOP/s",
                                      "peak": p64, "frac": fl / (sns * 1e-9) / 1e12 / p64,
                                      "peak_source": p64_src, "algorithmic_flops_per_launch": fl})
        line["peaks_measured_here"] = lp
        if fp64_value is not None:
            line["fp64_march"] = {"value": fp64_value, "unit": UNIT, "max_rel_l2_vs_oracle": fp64_err}
        print(json.dumps(line), flush=True)
    P.pe3d_destroy(plan)
    barrier()
    return 0


def run_batched(args):
    """32 frequencies, 25-400 Hz, on one 30 deg sector over 3000 m to 20 km, all
    marched in one batched persistent launch (complex FP32, FP64 setup).  The
    oracle marches the four lowest frequencies in full for parity and for the
    CPU baseline."""
    import torch
    import oracle
    from paper_1711_00005_gb300 import build
    build.build()
    import paper_1711_00005_gb300 as P
    grids = workloads.config4_grids()
    if args.members:                          # the highest-frequency members only (profiling cases)
        grids = grids[-args.members:]
    if args.range_steps:
        for g in grids:
            g.steps = min(g.steps, args.range_steps)
    for g in grids:
        g.stride = g.steps
    wls = [workloads.config4_member(g) for g in grids]
    point_steps = sum(g.point_steps for g in grids)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    plans, n2s, u0s, outs = [], [], [], []
    for wl in wls:
        g = wl.grid
        h = P.pe3d_plan(g.Nz, g.Ntheta, g.dz, g.dtheta, g.dr, g.k0, P.PE3D_WALLED, P.PE3D_FP32, stream)
        plans.append(h)
        n2s.append(torch.from_numpy(wl.n2).to(dev))
        u0s.append(torch.from_numpy(wl.u0.astype(np.complex64)).to(dev))
        outs.append(torch.empty((1, g.Ntheta, g.Nz), dtype=torch.complex64, device=dev))
    P.pe3d_set_option(plans[0], P.PE3D_OPT_TIMING, 1)
    torch.cuda.synchronize()

    def step():
        P.pe3d_set_medium_batched(plans, n2s, [wl.slice_r for wl in wls])
        P.pe3d_march_batched(plans, u0s, [g.r0 for g in grids], [g.steps for g in grids],
                             [g.stride for g in grids], outs)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # parity and CPU baseline: the four lowest frequencies, full marches
    cores = oracle.default_threads()
    err, t_cpu, ps_cpu = 0.0, 0.0, 0
    if not args.no_cpu_baseline:
        for i in range(min(4, len(wls))):
            ref, dt = oracle_run(wls[i], grids[i].steps, cores)
            got = outs[i].cpu().numpy()
            err = max(err, max(relerr_series(got, ref)))
            t_cpu += dt
            ps_cpu += grids[i].point_steps
    sampler = ClockSampler(gpu_uuid())
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    kernel_ns = []
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        step()
        kernel_ns.append(P.pe3d_plan_info(plans[0])["kernel_ns"])
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    t = ev0.elapsed_time(ev1) / 1e3
    peak, peak_kind = measured_peaks()
    kns = statistics.mean(kernel_ns) if kernel_ns and kernel_ns[0] > 0 else None
    roof = None
    if kns:
        achieved = 40 * point_steps / (kns * 1e-9) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": f"{peak_kind} hbm_gbs", "kernel": "k_march_batched<float2>",
                "algorithmic_bytes_per_launch": 40 * point_steps, "kernel_ms": kns / 1e6,
                "traffic": recorded_traffic("k_march_batched<float2>", "batched-32f-25-400Hz")}
    # end to end: host (pinned) media and starters through the same calls
    n2h = [torch.from_numpy(wl.n2).pin_memory() for wl in wls]
    u0h = [torch.from_numpy(wl.u0.astype(np.complex64)).pin_memory() for wl in wls]
    outh = [torch.empty((1, g.Ntheta, g.Nz), dtype=torch.complex64).pin_memory() for g in grids]
    t0 = time.perf_counter()
    P.pe3d_set_medium_batched(plans, n2h, [wl.slice_r for wl in wls])
    for u, ud in zip(u0h, u0s):
        ud.copy_(u, non_blocking=True)
    P.pe3d_march_batched(plans, u0s, [g.r0 for g in grids], [g.steps for g in grids],
                         [g.stride for g in grids], outs)
    for o, od in zip(outh, outs):
        o.copy_(od)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    line = {
        "metric": METRIC, "value": point_steps * args.steps / t, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batched-32f-25-400Hz", "marches": len(grids), "point_steps_per_launch": point_steps,
                   "range_steps": [grids[0].steps, grids[-1].steps],
                   "grid_range": [[grids[0].Nz, grids[0].Ntheta], [grids[-1].Nz, grids[-1].Ntheta]],
                   "precision": "complex64 march, FP64 coefficient setup", "exec": "one batched persistent launch",
                   "l2": "working set (fields and coefficients of 32 marches, ~0.6 GB) exceeds the 129 MB L2"},
        "max_rel_l2_vs_oracle": err if not args.no_cpu_baseline else None,
        "roofline": roof,
        "cpu_baseline": None if args.no_cpu_baseline else {
            "value": ps_cpu / t_cpu, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "full marches of the four lowest frequencies (25-29 Hz), FP64 C oracle"},
        "e2e": {"value": point_steps / t_e2e, "unit": UNIT,
                "h2d_bytes_per_step": int(sum(wl.n2.nbytes for wl in wls) + sum(u.numel() * 8 for u in u0h)),
                "d2h_bytes_per_step": int(sum(o.numel() * 8 for o in outh))},
        # per step: one depth set-up and one azimuth set-up for all marches, a prologue per
        # march, the batched march
        "gpu_launches": int(2 + len(plans) + 1) * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    for h in plans:
        P.pe3d_destroy(h)
    return 0


FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # 152 SMs x 128 FP32 lanes x FMA x 2.07 GHz


def run_broadband(args):
    """The paper's wide-band run (Sec. 4: 120 frequencies on one grid) at one-GPU
    size: 120 frequencies over 40-60 Hz on a 384 x 128 grid, 800 range steps,
    marched in one batched launch with pressure output, then the time series
    of every grid point at the last range (1024 samples) by pe3d_synthesize.
    The oracle marches every 15th frequency (8 of them, the paper's smaller
    case) for parity and for the CPU baseline, and re-synthesizes a sample of
    receivers from the GPU's pressures."""
    import torch
    import oracle
    from paper_1711_00005_gb300 import build
    build.build()
    import paper_1711_00005_gb300 as P
    bb = workloads.broadband()
    if args.range_steps:
        for wl in bb.members:
            wl.grid.steps = wl.grid.stride = min(wl.grid.steps, args.range_steps)
    grids = [wl.grid for wl in bb.members]
    g = grids[0]
    F, R = len(bb.members), g.points
    point_steps = sum(x.point_steps for x in grids)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    plans, u0s, outs = [], [], []
    n2 = torch.from_numpy(bb.members[0].n2).to(dev)          # one medium for every frequency
    for wl in bb.members:
        h = P.pe3d_plan(g.Nz, g.Ntheta, g.dz, g.dtheta, g.dr, wl.grid.k0, P.PE3D_WALLED, P.PE3D_FP32, stream)
        P.pe3d_set_option(h, P.PE3D_OPT_OUTPUT, P.PE3D_OUT_PRESSURE)
        plans.append(h)
        u0s.append(torch.from_numpy(wl.u0.astype(np.complex64)).to(dev))
        outs.append(torch.empty((1, g.Ntheta, g.Nz), dtype=torch.complex64, device=dev))
    P.pe3d_set_option(plans[0], P.PE3D_OPT_TIMING, 1)
    series = torch.empty((R, bb.T), dtype=torch.float32, device=dev)
    slice_r = bb.members[0].slice_r
    def step(timed_synthesis=None):
        P.pe3d_set_medium_batched(plans, [n2] * F, [slice_r] * F)
        P.pe3d_march_batched(plans, u0s, [x.r0 for x in grids], [x.steps for x in grids],
                             [x.stride for x in grids], outs)
        if timed_synthesis is not None:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
        P.pe3d_synthesize(P.PE3D_FP32, bb.freqs, bb.W, outs, bb.T, bb.t0, bb.dt, series, stream)
        if timed_synthesis is not None:
            b.record(stream)
            timed_synthesis.append((a, b))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    cores = oracle.default_threads()
    err, err_syn, t_cpu, ps_cpu = None, None, 0.0, 0
    if not args.no_cpu_baseline:
        err = 0.0
        for i in range(0, F, 15):
            wl = bb.members[i]
            ref, dt = oracle_run(wl, grids[i].steps, cores)
            p_ref = oracle.pressure(ref, oracle.snapshot_ranges(g.r0, g.dr, grids[i].steps, grids[i].stride),
                                    wl.grid.k0)
            err = max(err, max(relerr_series(outs[i].cpu().numpy(), p_ref)))
            t_cpu += dt
            ps_cpu += grids[i].point_steps
        rng = np.random.default_rng(0)
        pick = np.sort(rng.choice(R, size=min(R, 256), replace=False))
        p_gpu = np.array([o.cpu().numpy().reshape(-1)[pick] for o in outs])
        s_ref = oracle.synthesize(bb.freqs, bb.W, p_gpu, bb.t0, bb.dt, bb.T)
        got = series.cpu().numpy()[pick]
        err_syn = float(np.linalg.norm(got - s_ref) / np.linalg.norm(s_ref))
    sampler = ClockSampler(gpu_uuid())
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    kernel_ns, pairs = [], []
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        step(pairs)
        kernel_ns.append(P.pe3d_plan_info(plans[0])["kernel_ns"])
    ev1.record(stream)
    torch.cuda.synchronize()
    syn = [a.elapsed_time(b) for a, b in pairs]
    clocks = sampler.stop()
    t = ev0.elapsed_time(ev1) / 1e3
    peak, peak_kind = measured_peaks()
    kns = statistics.mean(kernel_ns) if kernel_ns and kernel_ns[0] > 0 else None
    roof = None
    if kns:
        achieved = 40 * point_steps / (kns * 1e-9) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": f"{peak_kind} hbm_gbs", "kernel": "k_march_batched<float2>",
                "algorithmic_bytes_per_launch": 40 * point_steps, "kernel_ms": kns / 1e6,
                "traffic": recorded_traffic("k_march_batched<float2>", g.name)}
    syn_ms = statistics.mean(syn)
    syn_flops = 4.0 * R * bb.T * F
    # end to end: host (pinned) medium, starters and series through the same calls
    n2h = torch.from_numpy(bb.members[0].n2).pin_memory()
    u0h = [torch.from_numpy(wl.u0.astype(np.complex64)).pin_memory() for wl in bb.members]
    sh = torch.empty((R, bb.T), dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    P.pe3d_set_medium_batched(plans, [n2h] * F, [slice_r] * F)
    with torch.cuda.stream(stream):
        for u, ud in zip(u0h, u0s):
            ud.copy_(u, non_blocking=True)
    P.pe3d_march_batched(plans, u0s, [x.r0 for x in grids], [x.steps for x in grids],
                         [x.stride for x in grids], outs)
    P.pe3d_synthesize(P.PE3D_FP32, bb.freqs, bb.W, outs, bb.T, bb.t0, bb.dt, series, stream)
    with torch.cuda.stream(stream):
        sh.copy_(series, non_blocking=True)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    line = {
        "metric": METRIC, "value": point_steps * args.steps / t, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": g.name, "frequencies": F, "band_hz": [float(bb.freqs[0]), float(bb.freqs[-1])],
                   "Nz": g.Nz, "Ntheta": g.Ntheta, "range_steps": g.steps, "point_steps_per_launch": point_steps,
                   "series": {"receivers": R, "samples": bb.T, "dt_s": bb.dt},
                   "precision": "complex64 march and synthesis, FP64 coefficients and phases",
                   "exec": "FP64 set-up of all frequencies in one launch each (depth, azimuth), batched "
                           "persistent launches of up to 64 marches, pe3d_synthesize",
                   "l2": "working set (120 marches' fields and coefficients, ~1.5 GB) exceeds the 129 MB L2"},
        "max_rel_l2_vs_oracle": err,
        "synthesis_rel_l2_vs_oracle": err_syn,
        "roofline": roof,
        "synthesis": {"ms": syn_ms, "kernels": "k_synth_phasors + k_synth<float2>", "bound": "alu",
                      "achieved": syn_flops / (syn_ms * 1e-3) / 1e12, "unit": "TFLOP/s", "peak": FP32_ALU_TFLOPS,
                      "frac": syn_flops / (syn_ms * 1e-3) / 1e12 / FP32_ALU_TFLOPS,
                      "peak_source": "FP32 FMA rate from unit counts and the 2.07 GHz maximum clock",
                      "algorithmic_flops": syn_flops},
        "cpu_baseline": None if args.no_cpu_baseline else {
            "value": ps_cpu / t_cpu, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "full marches of every 15th frequency (8 of 120), FP64 C oracle"},
        "e2e": {"value": point_steps / t_e2e, "unit": UNIT,
                "h2d_bytes_per_step": int(F * bb.members[0].n2.nbytes + sum(u.numel() * 8 for u in u0h)),
                "d2h_bytes_per_step": int(sh.numel() * 4)},
        # per step: one depth and one azimuth set-up for all frequencies, a prologue per
        # frequency, the batched march (64 marches per launch), two synthesis kernels
        "gpu_launches": int(2 + F + -(-F // 64) + 2) * args.steps,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    for h in plans:
        P.pe3d_destroy(h)
    return 0


def run_served(args):
    """The request loop under a Poisson stream (seed 5): f ~ U(25,400) Hz, sector
    width ~ U(10,360) deg, range ~ U(5,30) km; dz = lambda/8 over 1000 m,
    dr = lambda/4, Ntheta scaled with the width; one seeded medium slice per
    request (Munk + perturbations, generated at arrival).  Reports p50/p99
    submit-to-done latency, offered and served grid-point range-steps/s and the
    backlog left when the run stops."""
    import torch
    from paper_1711_00005_gb300 import build
    build.build()
    import paper_1711_00005_gb300 as P
    reqs = workloads.config5_stream(rate=args.serve_rate, duration=args.serve_duration, seed=5)
    grids = [workloads.config5_grid(r, max_steps=args.range_steps or None) for r in reqs]
    offered_ps = sum(g.point_steps for g in grids)
    srv = P.pe3d_server_create(int(args.serve_budget_gb * (1 << 30)), 64, args.serve_chunk)
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_uuid())
    t0 = time.perf_counter()
    pending = {}          # id -> (index, grid, keepalive)
    done = []             # (index, times)
    sample = {}           # index -> result (first few, for the alone-vs-mix check)
    i = 0
    deadline = args.serve_duration + args.serve_max_wait
    while True:
        now = time.perf_counter() - t0
        while i < len(reqs) and reqs[i].t_arrive <= now:
            wl = workloads.config5_member(reqs[i], grids[i], n_slices=1)
            req, keep = P.make_request(grids[i], wl.n2, wl.slice_r, wl.u0, fp32=True,
                                       out_stride=grids[i].steps, rc_every=args.serve_rc)
            rid = P.pe3d_submit(srv, req)
            pending[rid] = (i, grids[i], keep, wl)
            i += 1
        for rid in list(pending):
            st, tm = P.pe3d_poll(srv, rid)
            if st == P.PE3D_REQ_DONE:
                idx, g, keep, wl = pending.pop(rid)
                out = np.empty((1, g.Ntheta, g.Nz), np.complex64)
                P.pe3d_poll(srv, rid, out)
                done.append((idx, tm))
                if len(sample) < args.serve_check:
                    sample[idx] = (wl, out)
            elif st == P.PE3D_REQ_FAILED:
                raise RuntimeError(f"request {rid} failed")
        if i == len(reqs) and not pending:
            break
        if now > deadline:
            break
        time.sleep(0.001)
    wall = time.perf_counter() - t0
    clocks = sampler.stop()
    stats = P.pe3d_server_stats(srv)
    P.pe3d_server_destroy(srv)
    lat = sorted(tm[2] - tm[0] for _, tm in done)
    served_ps = sum(grids[idx].point_steps for idx, _ in done)
    t_first = min(tm[0] for _, tm in done) if done else 0.0
    t_last = max(tm[2] for _, tm in done) if done else 1.0
    # the same requests marched alone (pe3d_march) give bit-identical fields
    same = True
    for idx, (wl, out) in sample.items():
        g = grids[idx]
        with P.Plan.for_grid(g, fp32=True, exec_mode=P.PE3D_EXEC_PERSISTENT) as plan:
            if args.serve_rc:
                P.pe3d_set_option(plan.h, P.PE3D_OPT_RC_EVERY, args.serve_rc)
            plan.set_medium(wl.n2, wl.slice_r)
            ref = np.zeros((1, g.Ntheta, g.Nz), np.complex64)
            P.pe3d_march(plan.h, wl.u0.astype(np.complex64), g.r0, g.steps, g.steps, ref)
        same = same and bool(np.array_equal(out, ref))
    pct = lambda q: lat[min(len(lat) - 1, int(q * len(lat)))] if lat else None
    value = served_ps / (t_last - t_first) if done else 0.0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": len(done), "warmup": 0,
        "ms_per_step": (t_last - t_first) / max(1, len(done)) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"served-poisson-{args.serve_rate:g}rps-{args.serve_duration:g}s",
                   "requests_offered": len(reqs), "requests_done": len(done), "backlog_at_stop": len(pending),
                   "never_submitted": len(reqs) - i, "offered_point_steps": offered_ps,
                   "offered_point_steps_per_s": offered_ps / args.serve_duration,
                   "chunk_steps_per_tick": args.serve_chunk, "max_active": 64,
                   "precision": "complex64 march, FP64 coefficient setup"
                                + (f", FP64 residual correction every {args.serve_rc} steps" if args.serve_rc else ""),
                   "admission": "a thread of its own: each request is set up on its own stream, off the "
                                "batch's critical path",
                   "medium": "one seeded slice per request (Munk + perturbations)"},
        "latency_s": {"p50": pct(0.50), "p99": pct(0.99), "max": lat[-1] if lat else None},
        "alone_vs_mix_bitwise": same, "alone_vs_mix_checked": len(sample),
        "server_stats": stats, "wall_s": wall, "clocks": clocks,
        "gpu_busy_frac": (stats.get("kernel_us", 0) / 1e6 / wall) if wall > 0 else None,
        "roofline": None, "cpu_baseline": None,
        "e2e": {"value": value, "unit": UNIT, "note": "host media in, host fields out through pe3d_submit/poll"},
        "gpu_launches": stats.get("launches"),
    }
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + ["batched-25-400Hz", "broadband-120f", "served"],
                    default="medium-100Hz")
    ap.add_argument("--exec", type=int, default=0,
                    help="0 library choice (after --autotune-steps), 1 stream, 2 graph, 3 persistent, 4 resident")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--ref-sample-steps", type=int, default=200)
    ap.add_argument("--one-thread-steps", type=int, default=20,
                    help="range steps of the one-thread oracle sample beside the all-core baseline")
    ap.add_argument("--range-steps", type=int, default=0, help="truncate the march (profiling)")
    ap.add_argument("--rc", type=int, default=0, help="FP64 residual correction every K steps (FP32)")
    ap.add_argument("--output", choices=["field", "pressure", "tl"], default="field",
                    help="what the snapshots hold: the envelope, the pressure or the transmission loss")
    ap.add_argument("--members", type=int, default=0, help="batched workload: highest-frequency members only")
    ap.add_argument("--autotune-steps", type=int, default=100,
                    help="time candidate layouts over this many range steps before warm-up (0: off)")
    ap.add_argument("--serve-rate", type=float, default=200.0, help="served workload: Poisson arrivals per s")
    ap.add_argument("--serve-duration", type=float, default=60.0, help="served workload: seconds of arrivals")
    ap.add_argument("--serve-max-wait", type=float, default=120.0, help="served workload: stop this long after")
    ap.add_argument("--serve-chunk", type=int, default=64, help="served workload: range steps per tick")
    ap.add_argument("--serve-budget-gb", type=float, default=96.0, help="served workload: device memory budget")
    ap.add_argument("--serve-check", type=int, default=4, help="served workload: results re-marched alone")
    ap.add_argument("--serve-rc", type=int, default=64,
                    help="served workload: FP64 residual correction every K steps (0: off); 64 as specified")
    args = ap.parse_args(argv)
    args.warmup = max(3, args.warmup)     # timing rule: at least 3 untimed warm-up steps
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched-25-400Hz":
        return run_batched(args)
    if args.workload == "served":
        return run_served(args)
    if args.workload == "broadband-120f":
        return run_broadband(args)
    if args.rc and WORKLOADS[args.workload][0] != "fp32":
        ap.error("--rc applies to FP32 workloads")
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())

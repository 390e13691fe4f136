"""Python binding of libpe3d (the 3D wide-angle PE range march on GB300).

Thin ctypes marshalling over the C ABI declared in include/pe3d.h: every
function below has the C function's name and arguments, converts Python
objects (torch tensors on the GPU or CPU, numpy arrays) to pointers and
on-device flags, and raises PE3DError on a negative status.  All arithmetic
runs in the library's CUDA kernels; there is no Python or CPU path.  If the
shared object is missing, loading fails loudly.
"""
from __future__ import annotations

import ctypes
import os
from typing import Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpe3d.so")

PE3D_OK = 0
PE3D_ERR_ARG = -1
PE3D_ERR_OOM = -2
PE3D_ERR_SINGULAR = -3
PE3D_ERR_TIMEOUT = -4
PE3D_ERR_CUDA = -5
PE3D_ERR_STATE = -6
PE3D_ERR_BUSY = -7

PE3D_WALLED = 0
PE3D_PERIODIC = 1
PE3D_FP64 = 0
PE3D_FP32 = 1

PE3D_EXEC_AUTO = 0
PE3D_EXEC_STREAM = 1
PE3D_EXEC_GRAPH = 2
PE3D_EXEC_PERSISTENT = 3
PE3D_EXEC_RESIDENT = 4

PE3D_OPT_EXEC = 1
PE3D_OPT_ZTHREADS = 2
PE3D_OPT_TTILE = 3
PE3D_OPT_RC_EVERY = 4
PE3D_OPT_TIMING = 5
PE3D_OPT_OUTPUT = 6
PE3D_OPT_CTAS = 7
PE3D_OPT_Y_MIDPOINT = 8
PE3D_OPT_MEDIUM_INTERP = 9
PE3D_OPT_SCHEME = 10
PE3D_OPT_WAIT_LIMIT = 11
PE3D_SCHEME_PADE = 0
PE3D_SCHEME_TAYLOR = 1
PE3D_OUT_FIELD = 0
PE3D_OUT_PRESSURE = 1
PE3D_OUT_TL = 2

PE3D_REQ_PENDING = 0
PE3D_REQ_RUNNING = 1
PE3D_REQ_DONE = 2
PE3D_REQ_FAILED = 3

INFO_FIELDS = ("Nz", "Ntheta", "ldz", "zthreads", "zchunk", "ttile", "tchunk", "exec", "device_bytes",
               "launches", "grid", "kernel_ns", "total_launches", "setup_ns")


class PE3DError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pe3d error {code}: {msg}")
        self.code = code


class pe3d_request(ctypes.Structure):
    _fields_ = [("Nz", ctypes.c_int), ("Ntheta", ctypes.c_int),
                ("dz", ctypes.c_double), ("dtheta", ctypes.c_double), ("dr", ctypes.c_double),
                ("k0", ctypes.c_double), ("boundary", ctypes.c_int), ("precision", ctypes.c_int),
                ("rc_every", ctypes.c_int), ("n2", ctypes.c_void_p), ("slice_r", ctypes.c_void_p),
                ("K", ctypes.c_int), ("u0", ctypes.c_void_p), ("r0", ctypes.c_double),
                ("steps", ctypes.c_int), ("out_stride", ctypes.c_int)]


_lib = None

_SIGS = {
    "pe3d_plan": ([ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                   ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                   ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "pe3d_set_option": ([ctypes.c_void_p, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "pe3d_get_option": ([ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "pe3d_set_medium": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int],
                        ctypes.c_int),
    "pe3d_march": ([ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                    ctypes.c_int, ctypes.c_void_p, ctypes.c_int], ctypes.c_int),
    "pe3d_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "pe3d_plan_info": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_int], ctypes.c_int),
    "pe3d_autotune": ([ctypes.c_void_p, ctypes.c_double, ctypes.c_int], ctypes.c_int),
    "pe3d_march_batched": ([ctypes.c_int, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                            ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                            ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "pe3d_last_error": ([], ctypes.c_char_p),
    "pe3d_march_static": ([ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                           ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                           ctypes.c_int, ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                           ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "pe3d_set_medium_batched": ([ctypes.c_int, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                 ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_int), ctypes.c_int],
                                ctypes.c_int),
    "pe3d_synthesize": ([ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                         ctypes.POINTER(ctypes.c_void_p), ctypes.c_longlong, ctypes.c_int, ctypes.c_double,
                         ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p], ctypes.c_int),
    "pe3d_server_create": ([ctypes.c_size_t, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)],
                           ctypes.c_int),
    "pe3d_submit": ([ctypes.c_void_p, ctypes.POINTER(pe3d_request), ctypes.POINTER(ctypes.c_uint64)],
                    ctypes.c_int),
    "pe3d_poll": ([ctypes.c_void_p, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int), ctypes.c_void_p,
                   ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "pe3d_server_destroy": ([ctypes.c_void_p], ctypes.c_int),
    "pe3d_server_stats": ([ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.c_int], ctypes.c_int),
}


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libpe3d.so (built by build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1711_00005_gb300.build.build() "
                           "(there is no fallback path)")
    L = ctypes.CDLL(path)
    for name, (args, res) in _SIGS.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def _check(rc: int) -> int:
    if rc < 0:
        msg = load_library().pe3d_last_error().decode(errors="replace")
        raise PE3DError(rc, msg)
    return rc


def _ptr(x):
    """(pointer, on_device, keepalive) of a torch tensor, numpy array or None."""
    if x is None:
        return None, 0, None
    mod = type(x).__module__
    if mod.startswith("torch"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr()), int(x.is_cuda), x
    a = np.ascontiguousarray(x)
    return ctypes.c_void_p(a.ctypes.data), 0, a


def _stream_handle(stream) -> ctypes.c_void_p:
    if stream is None:
        return ctypes.c_void_p(None)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


# ----------------------------------------------------------------------------
# the C ABI, one function each
# ----------------------------------------------------------------------------

def pe3d_plan(Nz: int, Ntheta: int, dz: float, dtheta: float, dr: float, k0: float,
              boundary: int = PE3D_WALLED, precision: int = PE3D_FP64, cuda_stream=None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load_library().pe3d_plan(Nz, Ntheta, dz, dtheta, dr, k0, boundary, precision,
                                    _stream_handle(cuda_stream), ctypes.byref(h)))
    return h


def pe3d_set_option(plan, option: int, value: int) -> None:
    _check(load_library().pe3d_set_option(plan, option, value))


def pe3d_get_option(plan, option: int) -> int:
    v = ctypes.c_int()
    _check(load_library().pe3d_get_option(plan, option, ctypes.byref(v)))
    return v.value


def pe3d_set_medium(plan, n2, slice_r) -> None:
    p, on_dev, keep = _ptr(n2)
    r = np.ascontiguousarray(slice_r, dtype=np.float64)
    _check(load_library().pe3d_set_medium(plan, p, ctypes.c_void_p(r.ctypes.data), len(r), on_dev))
    del keep


def pe3d_march(plan, u0, r0: float, steps: int, out_stride: int, out) -> None:
    pu, du, ku = _ptr(u0)
    po, do, ko = _ptr(out)
    _check(load_library().pe3d_march(plan, pu, du, float(r0), int(steps), int(out_stride), po, do))
    del ku, ko


def pe3d_destroy(plan) -> None:
    _check(load_library().pe3d_destroy(plan))


def pe3d_plan_info(plan) -> dict:
    buf = (ctypes.c_int64 * len(INFO_FIELDS))()
    n = _check(load_library().pe3d_plan_info(plan, buf, len(INFO_FIELDS)))
    return {INFO_FIELDS[i]: int(buf[i]) for i in range(n)}


def pe3d_autotune(plan, r0: float, steps: int) -> None:
    _check(load_library().pe3d_autotune(plan, float(r0), int(steps)))


def pe3d_march_batched(plans: Sequence, u0s: Sequence, r0s: Sequence[float], steps: Sequence[int],
                       out_strides: Sequence[int], outs: Sequence) -> None:
    n = len(plans)
    P = (ctypes.c_void_p * n)(*[p.value if isinstance(p, ctypes.c_void_p) else p for p in plans])
    keep = []
    U = (ctypes.c_void_p * n)()
    O = (ctypes.c_void_p * n)()
    for i in range(n):
        pu, du, ku = _ptr(u0s[i])
        po, do, ko = _ptr(outs[i])
        if not du or (outs[i] is not None and not do):
            raise ValueError("pe3d_march_batched takes device tensors")
        U[i] = pu.value
        O[i] = po.value if po is not None else None
        keep += [ku, ko]
    R = (ctypes.c_double * n)(*[float(x) for x in r0s])
    S = (ctypes.c_int * n)(*[int(x) for x in steps])
    D = (ctypes.c_int * n)(*[int(x) for x in out_strides])
    _check(load_library().pe3d_march_batched(n, P, U, R, S, D, O))
    del keep


def pe3d_march_static(Nz: int, Ntheta: int, dz: float, dtheta: float, dr: float, k0: float, boundary: int,
                      precision: int, n2, slice_r, u0, r0: float, steps: int, out_stride: int, out,
                      cuda_stream=None) -> None:
    """The allocation-free march (device n2, u0 and out); see include/pe3d.h."""
    pn, _, kn = _ptr(n2)
    pu, _, ku = _ptr(u0)
    po, _, ko = _ptr(out)
    r = np.ascontiguousarray(slice_r, dtype=np.float64)
    _check(load_library().pe3d_march_static(Nz, Ntheta, dz, dtheta, dr, k0, boundary, precision, pn,
                                            ctypes.c_void_p(r.ctypes.data), len(r), pu, float(r0), int(steps),
                                            int(out_stride), po, _stream_handle(cuda_stream)))
    del kn, ku, ko


def pe3d_set_medium_batched(plans: Sequence, n2s: Sequence, slice_rs: Sequence) -> None:
    """pe3d_set_medium for several plans in one depth set-up launch; n2s all
    device tensors or all host arrays (see include/pe3d.h)."""
    n = len(plans)
    if len(n2s) != n or len(slice_rs) != n:
        raise ValueError("one medium and one slice-range array per plan")
    ptrs = [_ptr(x) for x in n2s]
    on_dev = {d for _, d, _ in ptrs}
    if len(on_dev) != 1:
        raise ValueError("media must be all on the device or all on the host")
    rs = [np.ascontiguousarray(r, dtype=np.float64) for r in slice_rs]
    Pl = (ctypes.c_void_p * n)(*[p.value if isinstance(p, ctypes.c_void_p) else p for p in plans])
    N2 = (ctypes.c_void_p * n)(*[p for p, _, _ in ptrs])
    RS = (ctypes.c_void_p * n)(*[r.ctypes.data for r in rs])
    KK = (ctypes.c_int * n)(*[len(r) for r in rs])
    _check(load_library().pe3d_set_medium_batched(n, Pl, N2, RS, KK, on_dev.pop()))
    del ptrs, rs


def pe3d_synthesize(precision: int, freqs, W, ps: Sequence, T: int, t0: float, dt: float, out,
                    cuda_stream=None) -> None:
    """Broadband synthesis out[r][k] = Re sum_i W[i] ps[i][r] e^{-2 pi i freqs[i] (t0 + k dt)}:
    ps are F device tensors of R complex values each, out a device real tensor
    [R][T] (see include/pe3d.h)."""
    f = np.ascontiguousarray(freqs, dtype=np.float64)
    w = np.ascontiguousarray(W, dtype=np.complex128)
    F = len(f)
    if len(w) != F or len(ps) != F:
        raise ValueError("freqs, W and ps must have one entry per frequency")
    R = ps[0].numel()
    if any(p.numel() != R or not p.is_contiguous() for p in ps):
        raise ValueError("every pressure tensor must be contiguous with R values")
    arr = (ctypes.c_void_p * F)(*[p.data_ptr() for p in ps])
    po, _, ko = _ptr(out)
    _check(load_library().pe3d_synthesize(int(precision), F, ctypes.c_void_p(f.ctypes.data),
                                          ctypes.c_void_p(w.ctypes.data), arr, int(R), int(T), float(t0),
                                          float(dt), po, _stream_handle(cuda_stream)))
    del ko


def pe3d_last_error() -> str:
    return load_library().pe3d_last_error().decode(errors="replace")


def pe3d_server_create(mem_budget: int, max_active: int, chunk: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load_library().pe3d_server_create(int(mem_budget), int(max_active), int(chunk), ctypes.byref(h)))
    return h


def pe3d_submit(server, req: pe3d_request) -> int:
    rid = ctypes.c_uint64()
    _check(load_library().pe3d_submit(server, ctypes.byref(req), ctypes.byref(rid)))
    return rid.value


def pe3d_poll(server, rid: int, out=None):
    """Returns (state, (t_submit, t_start, t_done))."""
    st = ctypes.c_int()
    times = (ctypes.c_double * 3)()
    po, do, ko = _ptr(out)
    if do:
        raise ValueError("pe3d_poll copies into host memory")
    _check(load_library().pe3d_poll(server, ctypes.c_uint64(rid), ctypes.byref(st), po, times))
    del ko
    return st.value, (times[0], times[1], times[2])


def pe3d_server_destroy(server) -> None:
    _check(load_library().pe3d_server_destroy(server))


def pe3d_server_stats(server) -> dict:
    keys = ("submitted", "admitted", "finished", "failed", "ticks", "point_steps", "device_bytes", "launches",
            "tick_us", "kernel_us")
    buf = (ctypes.c_int64 * len(keys))()
    n = _check(load_library().pe3d_server_stats(server, buf, len(keys)))
    return {keys[i]: int(buf[i]) for i in range(n)}


# ----------------------------------------------------------------------------
# convenience: a plan object (still marshalling only)
# ----------------------------------------------------------------------------

class Plan:
    """Owning wrapper of a pe3d plan; fields in and out as torch tensors."""

    def __init__(self, Nz, Ntheta, dz, dtheta, dr, k0, *, periodic=False, fp32=False, stream=None,
                 exec_mode=None, zthreads=None, ttile=None, output=None, ctas=None, y_midpoint=None,
                 interp=None, scheme=None):
        import torch
        self.torch = torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self.Nz, self.Ntheta = Nz, Ntheta
        self.fp32 = fp32
        self.cdtype = torch.complex64 if fp32 else torch.complex128
        self.h = pe3d_plan(Nz, Ntheta, dz, dtheta, dr, k0, PE3D_PERIODIC if periodic else PE3D_WALLED,
                           PE3D_FP32 if fp32 else PE3D_FP64, stream)
        if exec_mode is not None:
            pe3d_set_option(self.h, PE3D_OPT_EXEC, exec_mode)
        if zthreads is not None:
            pe3d_set_option(self.h, PE3D_OPT_ZTHREADS, zthreads)
        if ttile is not None:
            pe3d_set_option(self.h, PE3D_OPT_TTILE, ttile)
        if ctas is not None:
            pe3d_set_option(self.h, PE3D_OPT_CTAS, ctas)
        if y_midpoint is not None:
            pe3d_set_option(self.h, PE3D_OPT_Y_MIDPOINT, int(y_midpoint))
        if scheme is not None:
            pe3d_set_option(self.h, PE3D_OPT_SCHEME, int(scheme))
        if interp is not None:
            pe3d_set_option(self.h, PE3D_OPT_MEDIUM_INTERP, int(interp))
        self.output = PE3D_OUT_FIELD if output is None else output
        if output is not None:
            pe3d_set_option(self.h, PE3D_OPT_OUTPUT, output)

    @classmethod
    def for_grid(cls, grid, **kw):
        return cls(grid.Nz, grid.Ntheta, grid.dz, grid.dtheta, grid.dr, grid.k0, periodic=grid.periodic, **kw)

    def set_medium(self, n2, slice_r):
        pe3d_set_medium(self.h, n2, slice_r)

    def march(self, u0, r0, steps, stride, out=None):
        torch = self.torch
        n_out = steps // stride
        if out is None:
            dt = self.cdtype
            if self.output == PE3D_OUT_TL:     # transmission loss is real
                dt = torch.float32 if self.fp32 else torch.float64
            out = torch.empty((n_out, self.Ntheta, self.Nz), dtype=dt, device="cuda")
        pe3d_march(self.h, u0, r0, steps, stride, out if n_out > 0 else None)
        return out

    def info(self):
        return pe3d_plan_info(self.h)

    def close(self):
        if self.h is not None:
            pe3d_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def make_request(grid, n2, slice_r, u0, *, fp32=False, r0=None, steps=None, out_stride=None, rc_every=0):
    """A pe3d_request over host arrays (the arrays must outlive pe3d_submit,
    which copies them); returns (request, keepalive)."""
    n2a = np.ascontiguousarray(n2, dtype=np.complex128)
    sra = np.ascontiguousarray(slice_r, dtype=np.float64)
    u0a = np.ascontiguousarray(u0, dtype=np.complex64 if fp32 else np.complex128)
    steps = grid.steps if steps is None else steps
    req = pe3d_request(Nz=grid.Nz, Ntheta=grid.Ntheta, dz=grid.dz, dtheta=grid.dtheta, dr=grid.dr, k0=grid.k0,
                       boundary=PE3D_PERIODIC if grid.periodic else PE3D_WALLED,
                       precision=PE3D_FP32 if fp32 else PE3D_FP64, rc_every=rc_every,
                       n2=n2a.ctypes.data, slice_r=sra.ctypes.data, K=len(sra), u0=u0a.ctypes.data,
                       r0=grid.r0 if r0 is None else r0, steps=steps,
                       out_stride=(grid.stride if out_stride is None else out_stride))
    return req, (n2a, sra, u0a)

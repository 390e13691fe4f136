"""Measured roofline denominators on the current GPU (libpe3d_peaks.so).

    l2_copy_gbs(bytes, reps)  read+write bandwidth of an L2-resident copy
    fma_tflops(fp64)          FP64 or FP32 FMA throughput

The benchmark reports the range march against these beside the HBM copy
bandwidth of MEASURED_PEAKS.json: the 100 Hz and 200 Hz fields stay in L2, so
L2 bandwidth is their memory roofline, and the FP64 paths are bound by the
FP64 pipe.
"""
from __future__ import annotations

import ctypes

from . import build as _build

_lib = None


def _load() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _build.build()
        L = ctypes.CDLL(_build.PEAKS_LIB)
        L.pe3d_peak_l2_copy.argtypes = [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        L.pe3d_peak_l2_copy.restype = ctypes.c_int
        L.pe3d_peak_fma.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        L.pe3d_peak_fma.restype = ctypes.c_int
        _lib = L
    return _lib


def l2_copy_gbs(nbytes: int = 32 << 20, reps: int = 200) -> float:
    out = ctypes.c_double()
    if _load().pe3d_peak_l2_copy(int(nbytes), int(reps), ctypes.byref(out)) != 0:
        raise RuntimeError("L2 copy probe failed")
    return out.value


def fma_tflops(fp64: bool) -> float:
    out = ctypes.c_double()
    if _load().pe3d_peak_fma(int(bool(fp64)), ctypes.byref(out)) != 0:
        raise RuntimeError("FMA probe failed")
    return out.value


def measure() -> dict:
    """L2 copy bandwidth at 8 and 32 MB footprints (the larger is the peak),
    and the FP64 and FP32 FMA rates."""
    l2 = {f"{mb}MB": l2_copy_gbs(mb << 20, 400 if mb <= 8 else 100) for mb in (8, 32)}
    return {"l2_gbs": max(l2.values()), "l2_by_footprint_gbs": l2, "fp64_tflops": fma_tflops(True),
            "fp32_tflops": fma_tflops(False),
            "how": "pe3d_peak_l2_copy: L2-only loads/stores (.cg), each CTA copying its own slice back and "
                   "forth `reps` times in one launch of 4 x 512-thread CTAs per SM, read+write bytes; "
                   "pe3d_peak_fma: 8 independent FMA chains per thread, 8 x 256-thread CTAs per SM; "
                   "best of 5 (3) CUDA-event timings after a warm-up"}


if __name__ == "__main__":
    import json
    print(json.dumps(measure(), indent=1))

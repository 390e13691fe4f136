"""FP64 CPU oracle for the 3D wide-angle PE range march (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow, obviously correct
reference the CUDA library is checked against (paper Eq. 4-8, Fig. 2; the C
source states each reading taken).  Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import this package; the library never does.

Pinning status (what fixes each function other than itself): the tridiagonal
and cyclic solvers are pinned to LAPACK via numpy.linalg.solve and to the
circulant FFT solution; the step is pinned to a dense LU solve of the printed
Eq. 4 on tiny grids, to the closed-form discrete eigenmode multipliers, to
exact norm conservation, to reversibility, to the theta-uniform reduction and
to mirror symmetry (tests/test_oracle_pins.py); the interpolated medium to a
medium linear in range (tests/pins.py); the pressure/TL output to Hankel's
expansion and tabulated Bessel zeros (tests/test_oracle_output.py); the
broadband synthesis to a single-frequency closed form, the FFT on a uniform
frequency grid and the delay theorem (tests/test_oracle_synthesis.py).
No value printed in the
paper pins it: the paper prints no field values (parity to the paper's own
outputs is unpinned).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pe3d_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp"]


def build(src: str = _SRC, out: str = _LIB, extra: list[str] | None = None) -> str:
    """Compile the oracle with gcc (plain C99, no FMA contraction, OpenMP)."""
    cmd = ["gcc", *CFLAGS, *(extra or []), src, "-o", out, "-lm"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return out


def _needs_build(src: str, out: str) -> bool:
    return not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src)


class OracleLib:
    """Typed handle on one compiled oracle shared object."""

    def __init__(self, path: str):
        self.path = path
        L = ctypes.CDLL(path)
        P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
        L.oracle_tridiag_solve.argtypes = [I, P, P, P, P]
        L.oracle_cyclic_solve.argtypes = [I, P, P, P, P]
        L.oracle_step.argtypes = [I, I, D, D, D, D, D, I, P, P, I, I]
        L.oracle_march.argtypes = [I, I, D, D, D, D, I, P, P, I, P, D, I, I, P, I, I, I, I]
        L.oracle_penta_solve.argtypes = [I, P, P]
        for f in ("oracle_tridiag_solve", "oracle_cyclic_solve", "oracle_step", "oracle_march",
                  "oracle_penta_solve"):
            getattr(L, f).restype = I
        self.L = L

    @staticmethod
    def _c128(a):
        return np.ascontiguousarray(a, dtype=np.complex128)

    def tridiag_solve(self, sub, diag, sup, b):
        sub, diag, sup = self._c128(sub), self._c128(diag), self._c128(sup)
        x = self._c128(b).copy()
        rc = self.L.oracle_tridiag_solve(len(x), sub.ctypes.data, diag.ctypes.data,
                                         sup.ctypes.data, x.ctypes.data)
        if rc:
            raise RuntimeError(f"oracle_tridiag_solve failed ({rc})")
        return x

    def cyclic_solve(self, sub, diag, sup, b):
        sub, diag, sup = self._c128(sub), self._c128(diag), self._c128(sup)
        x = self._c128(b).copy()
        rc = self.L.oracle_cyclic_solve(len(x), sub.ctypes.data, diag.ctypes.data,
                                        sup.ctypes.data, x.ctypes.data)
        if rc:
            raise RuntimeError(f"oracle_cyclic_solve failed ({rc})")
        return x

    def penta_solve(self, bands, b):
        """Solve with the oracle's banded elimination: bands [n][5] hold row i's
        columns i-2 .. i+2."""
        bands = self._c128(bands)
        x = self._c128(b).copy()
        rc = self.L.oracle_penta_solve(len(x), bands.ctypes.data, x.ctypes.data)
        if rc:
            raise RuntimeError(f"oracle_penta_solve failed ({rc})")
        return x

    def step(self, u, n2, *, dz, dtheta, dr, k0, rstar, periodic, nthreads=1, taylor=False):
        u = self._c128(u).copy()
        n2 = self._c128(n2)
        Nt, Nz = u.shape
        rc = self.L.oracle_step(Nz, Nt, dz, dtheta, dr, k0, rstar, int(periodic),
                                n2.ctypes.data, u.ctypes.data, int(nthreads), int(bool(taylor)))
        if rc:
            raise RuntimeError(f"oracle_step failed ({rc})")
        return u

    def march(self, grid, n2, slice_r, u0, *, steps=None, stride=None, r0=None, nthreads=None,
              y_midpoint=False, interp=False, taylor=False):
        steps = grid.steps if steps is None else steps
        stride = grid.stride if stride is None else stride
        r0 = grid.r0 if r0 is None else r0
        nthreads = default_threads() if nthreads is None else nthreads
        n2 = self._c128(n2)
        slice_r = np.ascontiguousarray(slice_r, dtype=np.float64)
        u0 = self._c128(u0)
        Nt, Nz = u0.shape
        n_out = steps // stride
        out = np.zeros((max(n_out, 1), Nt, Nz), np.complex128)
        rc = self.L.oracle_march(Nz, Nt, grid.dz, grid.dtheta, grid.dr, grid.k0, int(grid.periodic),
                                 n2.ctypes.data, slice_r.ctypes.data, len(slice_r), u0.ctypes.data,
                                 float(r0), int(steps), int(stride), out.ctypes.data, int(nthreads),
                                 int(bool(y_midpoint)), int(bool(interp)), int(bool(taylor)))
        if rc:
            raise RuntimeError(f"oracle_march failed ({rc})")
        return out[:n_out]


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)))


def load() -> OracleLib:
    """Build (if stale) and load the oracle."""
    global _lib
    with _lock:
        if _lib is None:
            if _needs_build(_SRC, _LIB):
                build()
            _lib = OracleLib(_LIB)
        return _lib


def march_workload(wl, **kw):
    """Oracle march of a workloads.Workload."""
    return load().march(wl.grid, wl.n2, wl.slice_r, wl.u0, **kw)


# ---------------------------------------------------------------------------
# pressure and transmission loss (Sec. 2: p = u w(r) with w the Hankel
# function H0^(1)(k0 r); Fig. 2 forms p every step and writes TL)
# ---------------------------------------------------------------------------

def hankel0(x):
    """H0^(1)(x) = J0(x) + i Y0(x), the library routine (scipy.special.hankel1)
    serving as this step.  Pinned in tests/test_oracle_output.py against
    Hankel's large-argument expansion and the tabulated zeros of J0 and Y0."""
    from scipy.special import hankel1
    return hankel1(0, np.asarray(x, dtype=np.float64))


def snapshot_ranges(r0, dr, steps, stride):
    """Ranges of the stored snapshots: after step j the march is at
    r0 + (j+1) dr, and snapshot s (1-based) is taken after step s*stride - 1."""
    n_out = steps // stride
    return r0 + dr * stride * np.arange(1, n_out + 1, dtype=np.float64)


def pressure(u_snaps, ranges, k0):
    """p = u H0^(1)(k0 r) for snapshots u_snaps[s] taken at ranges[s]."""
    h = hankel0(k0 * np.asarray(ranges, dtype=np.float64))
    return np.asarray(u_snaps, dtype=np.complex128) * h[:, None, None]


def transmission_loss(p):
    """TL = -20 log10 |p| in dB (Fig. 2, Fig. 5)."""
    return -20.0 * np.log10(np.abs(p))


# ---------------------------------------------------------------------------
# broadband synthesis.  The paper runs the march once per frequency of a
# wide-band signal (Fig. 1, the loop over frequencies; the 8- and
# 120-frequency tests of Sec. 4) but does not write out how the time signal is
# formed.  Reading taken: with the e^{-i w t} convention under which
# H0^(1)(k0 r) is outgoing, a receiver's time series is the sum over the
# computed frequencies s(t) = Re sum_i W_i p_i e^{-2 pi i f_i t}, W_i being the
# source spectrum times the frequency-quadrature weight.
# ---------------------------------------------------------------------------

def synthesize(freqs, W, p, t0, dt, T):
    """s[r][k] = Re sum_i W[i] p[i][r] exp(-2 pi i freqs[i] (t0 + k dt)) for
    p of shape [F][R]: one frequency at a time, in FP64."""
    freqs = np.asarray(freqs, dtype=np.float64)
    W = np.asarray(W, dtype=np.complex128)
    p = np.asarray(p, dtype=np.complex128).reshape(len(freqs), -1)
    t = t0 + dt * np.arange(T, dtype=np.float64)
    s = np.zeros((p.shape[1], T), np.float64)
    for i in range(len(freqs)):
        s += (W[i] * p[i][:, None] * np.exp(-2j * np.pi * freqs[i] * t[None, :])).real
    return s

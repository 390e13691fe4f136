"""Seeded synthetic inputs for the 3D wide-angle PE range march.

This module produces the *inputs* of a march -- the grid, the complex
refractive-index-squared field n^2(r, theta, z) sampled as range slices, and
the starting field u0 -- for the five workloads the project measures.  It
holds none of the marching scheme's arithmetic (no X or Y operator, no
tridiagonal system, no step): both the FP64 CPU oracle and the CUDA library
consume what it returns, and neither is imported here.

Grid conventions (shared by every consumer):

* depth points z_l = (l + 1) * dz, l = 0 .. Nz-1; Dirichlet ghosts at z = 0
  (pressure-release surface) and z = (Nz + 1) * dz (below the absorbing layer);
* walled sector: theta_m = theta_lo + (m + 1) * dtheta, walls at theta_lo and
  theta_lo + (Ntheta + 1) * dtheta; periodic: theta_m = m * dtheta with
  dtheta = 2 pi / Ntheta;
* the medium is piecewise constant in range: slice k, sampled at range R_k,
  is active for R_k <= r < R_{k+1}.

The paper (Sec. 4.1) measures a 50 Hz source at 100 m depth in a range-
independent ocean on data that is not available; every field below is a
seeded stand-in with the shapes and structure of the paper's 3D case, built
from the sound speed via n^2 = (c0 / c)^2 with c0 = 1500 m/s.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

C0 = 1500.0  # reference sound speed [m/s]; k0 = 2 pi f / C0


@dataclass
class Grid:
    """One march's grid and schedule (all lengths in metres, angles in rad)."""

    Nz: int
    Ntheta: int
    dz: float
    dtheta: float
    dr: float
    k0: float
    r0: float
    steps: int
    stride: int
    periodic: bool
    theta_lo: float = 0.0
    freq: float = 0.0
    name: str = ""

    @property
    def z(self) -> np.ndarray:
        return (np.arange(self.Nz) + 1.0) * self.dz

    @property
    def theta(self) -> np.ndarray:
        if self.periodic:
            return np.arange(self.Ntheta) * self.dtheta
        return self.theta_lo + (np.arange(self.Ntheta) + 1.0) * self.dtheta

    @property
    def points(self) -> int:
        return self.Nz * self.Ntheta

    @property
    def point_steps(self) -> int:
        return self.Nz * self.Ntheta * self.steps

    @property
    def n_out(self) -> int:
        return self.steps // self.stride if self.stride > 0 else 0


@dataclass
class Workload:
    grid: Grid
    slice_r: np.ndarray          # [K] ascending slice start ranges
    n2: np.ndarray               # [K][Ntheta][Nz] complex128
    u0: np.ndarray               # [Ntheta][Nz] complex128
    meta: dict = field(default_factory=dict)


# ----------------------------------------------------------------------------
# sound-speed building blocks
# ----------------------------------------------------------------------------

def munk(z: np.ndarray) -> np.ndarray:
    """Canonical Munk profile, axis at 1300 m."""
    eta = 2.0 * (z - 1300.0) / 1300.0
    return 1500.0 * (1.0 + 0.00737 * (eta - 1.0 + np.exp(-eta)))


class FourierPerturbation:
    """Gaussian random field by random Fourier features.

    dc(x, y, z) = sigma * sqrt(2/M) * sum_k cos(kappa_k . (x, y, z) + phi_k),
    kappa_k ~ N(0, ell^-2 I_3), phi_k ~ U(0, 2 pi), drawn from
    numpy.random.default_rng(seed) in that order (kappa first, then phi).
    Evaluated on a (theta, z) slice at range r as one complex matrix product,
    because cos(a + b + phi) = Re(exp(i(a + phi)) exp(i b)).
    """

    def __init__(self, seed: int, sigma: float, ell: float, M: int = 256):
        rng = np.random.default_rng(seed)
        self.kappa = rng.normal(0.0, 1.0 / ell, size=(M, 3))
        self.phi = rng.uniform(0.0, 2.0 * math.pi, size=M)
        self.amp = sigma * math.sqrt(2.0 / M)

    def slice(self, r: float, theta: np.ndarray, z: np.ndarray) -> np.ndarray:
        x = r * np.cos(theta)
        y = r * np.sin(theta)
        ph_t = np.outer(x, self.kappa[:, 0]) + np.outer(y, self.kappa[:, 1]) + self.phi[None, :]
        ph_z = np.outer(z, self.kappa[:, 2])
        return self.amp * (np.exp(1j * ph_t) @ np.exp(1j * ph_z).T).real


def _absorber(z: np.ndarray, z_top: float, z_bot: float, peak: float = 0.01) -> np.ndarray:
    """Im(n^2) rising quadratically from 0 at z_top to `peak` at z_bot."""
    t = np.clip((z - z_top) / (z_bot - z_top), 0.0, None)
    return peak * t * t


def _n2(c: np.ndarray, im: np.ndarray) -> np.ndarray:
    return (C0 / c) ** 2 + 1j * im


def slice_ranges(r0: float, steps: int, dr: float, spacing: float) -> np.ndarray:
    """Slice start ranges R_k = r0 + k * spacing covering (r0, r0 + steps*dr]."""
    r_end = r0 + steps * dr
    K = int(math.floor((r_end - r0) / spacing + 1e-9)) + 1
    return r0 + spacing * np.arange(K)


def gaussian_starter(grid: Grid, zs: float = 100.0, hann: bool | None = None, image: bool = False) -> np.ndarray:
    """Gaussian starter sqrt(k0) exp(-k0^2 (z - zs)^2 / 2), times a Hann taper
    sin^2(pi (m+1) / (Ntheta+1)) across a walled sector (uniform for 360 deg).
    With image, the source's mirror image in the pressure-release surface is
    subtracted, sqrt(k0) [exp(-k0^2 (z - zs)^2 / 2) - exp(-k0^2 (z + zs)^2 / 2)],
    so the starter vanishes at z = 0 as the field does."""
    k0 = grid.k0
    gz = math.sqrt(k0) * np.exp(-(k0 * k0) * (grid.z - zs) ** 2 / 2.0)
    if image:
        gz = gz - math.sqrt(k0) * np.exp(-(k0 * k0) * (grid.z + zs) ** 2 / 2.0)
    if hann is None:
        hann = not grid.periodic
    if hann:
        m = np.arange(grid.Ntheta)
        gt = np.sin(math.pi * (m + 1.0) / (grid.Ntheta + 1.0)) ** 2
    else:
        gt = np.ones(grid.Ntheta)
    return (gt[:, None] * gz[None, :]).astype(np.complex128)


def round32(x: float) -> int:
    return max(32, int(32 * round(x / 32.0)))


# ----------------------------------------------------------------------------
# the five measured workloads
# ----------------------------------------------------------------------------

def config1() -> Workload:
    """Plain FP64 march, walled 20 deg sector, 50 Hz, Nz=200 x Ntheta=64, 100 steps.

    Water 0-400 m at c = 1500 + dc (seed 0, sigma 2 m/s, ell 50 m); bottom
    400-500 m at 1700 m/s with Im(n^2) = 0.01 ((z-400)/100)^2.  One medium slice
    per range step.  Output every 10th step.
    """
    f = 50.0
    k0 = 2 * math.pi * f / C0
    Nz, Nt = 200, 64
    sector = math.radians(20.0)
    g = Grid(Nz=Nz, Ntheta=Nt, dz=2.5, dtheta=sector / (Nt + 1), dr=10.0, k0=k0,
             r0=100.0, steps=100, stride=10, periodic=False, theta_lo=-sector / 2,
             freq=f, name="walled-50Hz-200x64-100steps")
    pert = FourierPerturbation(seed=0, sigma=2.0, ell=50.0)
    z, th = g.z, g.theta
    R = g.r0 + g.dr * np.arange(g.steps)          # slice k active for step k
    n2 = np.empty((len(R), Nt, Nz), np.complex128)
    water = z <= 400.0
    for k, r in enumerate(R):
        c = np.where(water[None, :], 1500.0 + pert.slice(r, th, z), 1700.0)
        im = np.where(water, 0.0, 0.01 * ((z - 400.0) / 100.0) ** 2)
        n2[k] = _n2(c, np.broadcast_to(im, c.shape))
    return Workload(g, R, n2, gaussian_starter(g), {"seed": 0})


def _config2_grid() -> Grid:
    f = 100.0
    k0 = 2 * math.pi * f / C0
    Nz, Nt = 1067, 256
    sector = math.radians(45.0)
    return Grid(Nz=Nz, Ntheta=Nt, dz=1.875, dtheta=sector / (Nt + 1), dr=5.0, k0=k0,
                r0=100.0, steps=2000, stride=100, periodic=False, theta_lo=-sector / 2,
                freq=f, name="walled-100Hz-1067x256-2000steps")


def config2(steps: int | None = None, spacing: float = 100.0) -> Workload:
    """Medium single-frequency case: 100 Hz, 45 deg walled sector, Nz=1067 x Ntheta=256,
    dr = 5 m, 2000 steps (10 km).

    Munk profile plus seed-1 perturbations (sigma 2 m/s, ell 50 m) in the water;
    a planar sloping bottom D(r, theta) = 200 + 0.1 r cos(theta) (200 m to 1200 m
    over 10 km along theta = 0) with 1700 m/s sediment below it; an absorbing
    layer over the grid's bottom 20 % (1600-2000 m).  Slices every 100 m.
    """
    g = _config2_grid()
    if steps is not None:
        g.steps = steps
        g.stride = max(1, min(g.stride, steps))
    pert = FourierPerturbation(seed=1, sigma=2.0, ell=50.0)
    R = slice_ranges(g.r0, g.steps, g.dr, spacing)
    z, th = g.z, g.theta
    cz = munk(z)
    im = _absorber(z, 1600.0, 2000.0)
    n2 = np.empty((len(R), g.Ntheta, g.Nz), np.complex128)
    for k, r in enumerate(R):
        D = 200.0 + 0.1 * r * np.cos(th)
        c = cz[None, :] + pert.slice(r, th, z)
        c = np.where(z[None, :] > D[:, None], 1700.0, c)
        n2[k] = _n2(c, np.broadcast_to(im, c.shape))
    return Workload(g, R, n2, gaussian_starter(g), {"seed": 1, "slice_spacing": spacing})


def config3(steps: int | None = None, spacing: float = 100.0) -> Workload:
    """Full-360 deg periodic case: 200 Hz, Nz=1067 (dz = 0.9375 m over 1000 m) x
    Ntheta=1024, dr = 2.5 m, 4000 steps.  Munk background plus a mesoscale eddy
    dc = 20 exp(-|xy - xy0|^2 / (5 km)^2 - (z - 300)^2 / (300 m)^2) with its centre
    uniform over a 10 km disk from seed 2; absorbing layer over the bottom 200 m.
    """
    f = 200.0
    k0 = 2 * math.pi * f / C0
    Nz, Nt = 1067, 1024
    g = Grid(Nz=Nz, Ntheta=Nt, dz=0.9375, dtheta=2 * math.pi / Nt, dr=2.5, k0=k0,
             r0=100.0, steps=4000 if steps is None else steps, stride=200, periodic=True,
             freq=f, name="periodic-200Hz-1067x1024-4000steps")
    g.stride = max(1, min(g.stride, g.steps))
    rng = np.random.default_rng(2)
    rad = 10000.0 * math.sqrt(rng.uniform())
    ang = 2 * math.pi * rng.uniform()
    x0, y0 = rad * math.cos(ang), rad * math.sin(ang)
    R = slice_ranges(g.r0, g.steps, g.dr, spacing)
    z, th = g.z, g.theta
    cz = munk(z)
    im = _absorber(z, 800.0, 1000.0)
    ez = np.exp(-((z - 300.0) / 300.0) ** 2)
    n2 = np.empty((len(R), Nt, Nz), np.complex128)
    for k, r in enumerate(R):
        x, y = r * np.cos(th), r * np.sin(th)
        exy = np.exp(-((x - x0) ** 2 + (y - y0) ** 2) / 5000.0 ** 2)
        c = cz[None, :] + 20.0 * exy[:, None] * ez[None, :]
        n2[k] = _n2(c, np.broadcast_to(im, c.shape))
    return Workload(g, R, n2, gaussian_starter(g), {"seed": 2, "eddy_xy": (x0, y0)})


def config4_grids(max_range: float = 20000.0) -> list[Grid]:
    """Batched multi-frequency launch: 32 frequencies log-spaced 25-400 Hz on one
    30 deg walled sector over a 3000 m water column; dz = lambda/8,
    Ntheta = round32(128 sqrt(f / 25)), dr = lambda/4, marched to 20 km."""
    grids = []
    sector = math.radians(30.0)
    for i in range(32):
        f = 25.0 * 16.0 ** (i / 31.0)
        lam = C0 / f
        dz = lam / 8.0
        Nz = int(math.ceil(3000.0 / dz - 1e-9))
        Nt = round32(128.0 * math.sqrt(f / 25.0))
        dr = lam / 4.0
        steps = int(math.ceil(max_range / dr - 1e-9))
        grids.append(Grid(Nz=Nz, Ntheta=Nt, dz=dz, dtheta=sector / (Nt + 1), dr=dr,
                          k0=2 * math.pi * f / C0, r0=100.0, steps=steps,
                          stride=max(1, steps // 10), periodic=False, theta_lo=-sector / 2,
                          freq=f, name=f"batched-{f:.1f}Hz"))
    return grids


def config4_member(grid: Grid, seed: int = 3, spacing: float = 2500.0) -> Workload:
    """Medium of one config-4 frequency: Munk + seed-3 perturbations (sigma 2 m/s,
    ell 50 m), absorbing layer over the bottom 20 % (2400-3000 m), slices every
    `spacing` metres of range."""
    pert = FourierPerturbation(seed=seed, sigma=2.0, ell=50.0)
    R = slice_ranges(grid.r0, grid.steps, grid.dr, spacing)
    z, th = grid.z, grid.theta
    cz = munk(z)
    im = _absorber(z, 2400.0, 3000.0)
    n2 = np.empty((len(R), grid.Ntheta, grid.Nz), np.complex128)
    for k, r in enumerate(R):
        c = cz[None, :] + pert.slice(r, th, z)
        n2[k] = _n2(c, np.broadcast_to(im, c.shape))
    return Workload(grid, R, n2, gaussian_starter(grid), {"seed": seed, "slice_spacing": spacing})


@dataclass
class Request:
    idx: int
    t_arrive: float
    freq: float
    width_deg: float
    max_range: float


def config5_stream(rate: float = 200.0, duration: float = 60.0, seed: int = 5) -> list[Request]:
    """Poisson request stream: exponential inter-arrivals (mean 1/rate), then per
    request f ~ U(25, 400) Hz, sector width ~ U(10, 360) deg and max range
    ~ U(5, 30) km, drawn from default_rng(seed) in that order."""
    rng = np.random.default_rng(seed)
    out, t, i = [], 0.0, 0
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration:
            break
        f = rng.uniform(25.0, 400.0)
        w = rng.uniform(10.0, 360.0)
        rmax = rng.uniform(5000.0, 30000.0)
        out.append(Request(i, t, f, w, rmax))
        i += 1
    return out


def config5_grid(req: Request, depth: float = 1000.0, max_steps: int | None = None) -> Grid:
    """Grid of one served request: dz = lambda/8 over 1000 m, dr = lambda/4,
    Ntheta = max(32, round32(1024 * width / 360)); a width above 350 deg is
    served as the full periodic circle, narrower sectors are walled."""
    lam = C0 / req.freq
    dz, dr = lam / 8.0, lam / 4.0
    Nz = int(math.ceil(depth / dz - 1e-9))
    periodic = req.width_deg > 350.0
    width = 360.0 if periodic else req.width_deg
    Nt = max(32, round32(1024.0 * width / 360.0))
    steps = int(math.ceil(req.max_range / dr - 1e-9))
    if max_steps is not None:
        steps = min(steps, max_steps)
    sector = math.radians(width)
    return Grid(Nz=Nz, Ntheta=Nt, dz=dz,
                dtheta=(2 * math.pi / Nt) if periodic else sector / (Nt + 1),
                dr=dr, k0=2 * math.pi * req.freq / C0, r0=100.0, steps=steps,
                stride=steps, periodic=periodic, theta_lo=-sector / 2, freq=req.freq,
                name=f"req{req.idx}")


def config5_member(req: Request, grid: Grid, n_slices: int = 8) -> Workload:
    """Medium of one served request: Munk + perturbations seeded 1000 + idx,
    absorbing layer over the bottom 20 %, `n_slices` equal range slices."""
    pert = FourierPerturbation(seed=1000 + req.idx, sigma=2.0, ell=50.0, M=64)
    span = grid.steps * grid.dr
    R = grid.r0 + (span / n_slices) * np.arange(n_slices)
    z, th = grid.z, grid.theta
    cz = munk(z)
    im = _absorber(z, 800.0, 1000.0)
    n2 = np.empty((n_slices, grid.Ntheta, grid.Nz), np.complex128)
    for k, r in enumerate(R):
        c = cz[None, :] + pert.slice(r, th, z)
        n2[k] = _n2(c, np.broadcast_to(im, c.shape))
    return Workload(grid, R, n2, gaussian_starter(grid), {"seed": 1000 + req.idx})


# ----------------------------------------------------------------------------
# small randomised inputs for property and parity tests
# ----------------------------------------------------------------------------

def random_case(Nz: int, Ntheta: int, *, periodic: bool, K: int = 1, steps: int = 5,
                seed: int = 0, lossy: bool = True, theta_dependent: bool = True,
                k0: float = 0.4, dz: float = 2.0, dr: float = 5.0, r0: float = 100.0,
                dtheta: float | None = None, stride: int = 1) -> Workload:
    """A small seeded march with a rough, optionally lossy and theta-dependent
    medium (n^2 within [0.8, 1.1] + i [0, 0.02]) and a random complex start."""
    rng = np.random.default_rng(seed)
    if dtheta is None:
        dtheta = (2 * math.pi / Ntheta) if periodic else math.radians(20.0) / (Ntheta + 1)
    g = Grid(Nz=Nz, Ntheta=Ntheta, dz=dz, dtheta=dtheta, dr=dr, k0=k0, r0=r0,
             steps=steps, stride=stride, periodic=periodic, theta_lo=-0.1, name="random")
    shape = (K, Ntheta if theta_dependent else 1, Nz)
    re = rng.uniform(0.8, 1.1, size=shape)
    im = rng.uniform(0.0, 0.02, size=shape) if lossy else np.zeros(shape)
    n2 = np.broadcast_to(re + 1j * im, (K, Ntheta, Nz)).astype(np.complex128)
    span = max(steps * dr, 1.0)
    R = r0 + (span / K) * np.arange(K)
    u0 = rng.normal(size=(Ntheta, Nz)) + 1j * rng.normal(size=(Ntheta, Nz))
    return Workload(g, R, np.ascontiguousarray(n2), u0.astype(np.complex128), {"seed": seed})


def range_linear_case(Nz: int, Ntheta: int, *, periodic: bool, steps: int = 9, seed: int = 0,
                      slice_steps=(2.5, 4.2, 6.0), k0: float = 0.4, dz: float = 2.0, dr: float = 5.0,
                      r0: float = 100.0, dtheta: float | None = None, stride: int = 1) -> Workload:
    """Slices that sample a medium linear in range, n^2(r) = A + B (r - r0),
    at the non-uniform ranges r0 + slice_steps[k] dr.  A is rough and lossy
    (real part in [0.85, 1.05], imaginary in [0.005, 0.02]), B moves n^2 by at
    most 0.05 in real part and 0.004 in imaginary part over the slices' span.
    meta holds A and B."""
    rng = np.random.default_rng(seed)
    if dtheta is None:
        dtheta = (2 * math.pi / Ntheta) if periodic else math.radians(20.0) / (Ntheta + 1)
    g = Grid(Nz=Nz, Ntheta=Ntheta, dz=dz, dtheta=dtheta, dr=dr, k0=k0, r0=r0,
             steps=steps, stride=stride, periodic=periodic, theta_lo=-0.1, name="range-linear")
    shape = (Ntheta, Nz)
    A = rng.uniform(0.85, 1.05, size=shape) + 1j * rng.uniform(0.005, 0.02, size=shape)
    span = max(slice_steps[-1] * dr, 1.0)
    B = (rng.uniform(-0.05, 0.05, size=shape) + 1j * rng.uniform(-0.004, 0.004, size=shape)) / span
    R = r0 + dr * np.asarray(slice_steps, dtype=np.float64)
    n2 = np.stack([A + B * (r - r0) for r in R]).astype(np.complex128)
    u0 = rng.normal(size=shape) + 1j * rng.normal(size=shape)
    return Workload(g, R, np.ascontiguousarray(n2), u0.astype(np.complex128), {"seed": seed, "A": A, "B": B})


@dataclass
class Broadband:
    """A wide-band source marched once per frequency on one shared grid, and the
    synthesis parameters of its time series at the last range."""
    members: list            # Workload per frequency (same grid but k0)
    freqs: np.ndarray        # [F] Hz
    W: np.ndarray            # [F] complex: source spectrum times the frequency step
    t0: float                # first sample time [s]
    dt: float                # sample spacing [s]
    T: int                   # samples


def broadband(F: int = 120, f_lo: float = 40.0, f_hi: float = 60.0, *, Nz: int = 384, Ntheta: int = 128,
              steps: int = 800, T: int = 1024, slice_spacing: float = 500.0) -> Broadband:
    """The paper's wide-band runs (Sec. 4: 8 and 120 frequencies on one grid)
    at a size one GPU steps through in a fraction of a second.

    F frequencies uniform over [f_lo, f_hi]; one grid resolving f_hi
    (dz = lambda/8 at f_hi, 3.125 m for 60 Hz; dr = lambda/4, 6.25 m; 30 deg
    walled sector), r0 = 100 m, `steps` range steps (5 km at 800).  The medium
    is the walled 100 Hz case's kind at depth Nz*dz: Munk profile with seed-3
    perturbations (sigma 2 m/s, ell 50 m), a planar bottom D = 200 + 0.1 r
    cos(theta) with 1700 m/s below it and an absorbing bottom 20 % of the grid,
    one slice every `slice_spacing` m; it does not depend on frequency.  Each
    member starts from the Gaussian starter at its own k0.  The source spectrum
    is a Hann window over the band; W_i is it times the frequency step.  The
    series has T samples at 200 Hz (above twice f_hi), starting 1 s before the
    arrival time r_end / C0 at the last range."""
    freqs = np.linspace(f_lo, f_hi, F) if F > 1 else np.array([0.5 * (f_lo + f_hi)])
    lam = C0 / f_hi
    dz, dr = lam / 8.0, lam / 4.0
    sector = math.radians(30.0)
    g0 = Grid(Nz=Nz, Ntheta=Ntheta, dz=dz, dtheta=sector / (Ntheta + 1), dr=dr, k0=0.0, r0=100.0,
              steps=steps, stride=steps, periodic=False, theta_lo=-sector / 2, name="broadband")
    pert = FourierPerturbation(seed=3, sigma=2.0, ell=50.0)
    R = slice_ranges(g0.r0, steps, dr, slice_spacing)
    z, th = g0.z, g0.theta
    depth = Nz * dz
    cz = munk(z)
    im = _absorber(z, 0.8 * depth, depth)
    n2 = np.empty((len(R), Ntheta, Nz), np.complex128)
    for k, r in enumerate(R):
        D = 200.0 + 0.1 * r * np.cos(th)
        c = cz[None, :] + pert.slice(r, th, z)
        c = np.where(z[None, :] > D[:, None], 1700.0, c)
        n2[k] = _n2(c, np.broadcast_to(im, c.shape))
    members = []
    for f in freqs:
        g = Grid(**{**g0.__dict__, "k0": 2 * math.pi * f / C0, "freq": float(f),
                    "name": f"broadband-{F}f-{f_lo:g}-{f_hi:g}Hz-{Nz}x{Ntheta}-{steps}steps"})
        members.append(Workload(g, R, n2, gaussian_starter(g), {"seed": 3}))
    df = (f_hi - f_lo) / (F - 1) if F > 1 else 1.0
    hann = np.sin(np.pi * (freqs - f_lo) / (f_hi - f_lo)) ** 2 if F > 1 else np.ones(1)
    W = (hann * df).astype(np.complex128)
    r_end = g0.r0 + steps * dr
    return Broadband(members, freqs, W, r_end / C0 - 1.0, 1.0 / 200.0, T)

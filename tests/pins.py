"""Independent pins for the FP64 oracle.

Each check returns an error figure (relative, max over entries) so the same
functions serve the pin tests (error below tolerance) and the mutation test
(a planted mistake drives at least one of them above tolerance).  Nothing
here calls the CUDA library, and nothing re-types the oracle's loops: the
checks use LAPACK (numpy.linalg.solve) on dense matrices assembled from the
printed Eq. 4, closed-form eigenvalues of the discrete operators, the FFT of
a circulant matrix, and exact invariants of the scheme.
"""
from __future__ import annotations

import math

import numpy as np

import workloads

TOL = 1e-12


def relerr(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    den = max(np.linalg.norm(b.ravel()), 1e-300)
    return float(np.linalg.norm((a - b).ravel()) / den)


# --------------------------------------------------------------------------
# dense Eq. 4 (brute force on tiny grids)
# --------------------------------------------------------------------------

def second_difference(n: int, periodic: bool) -> np.ndarray:
    """The 3-point matrix tridiag(1, -2, 1), with wrap-around corners if periodic."""
    D = -2.0 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1)
    if periodic and n > 1:
        D[0, -1] += 1.0
        D[-1, 0] += 1.0
    return D


def dense_operators(n2_slice, grid, rstar):
    """X and Y of Eq. 4 as dense matrices on the vector u[m][l] -> m*Nz + l."""
    Nt, Nz = n2_slice.shape
    k0 = grid.k0
    s = 1.0 / (k0 * grid.dz) ** 2
    c = 1.0 / (k0 * rstar * grid.dtheta) ** 2
    Dz = second_difference(Nz, periodic=False)
    Dt = second_difference(Nt, periodic=grid.periodic)
    X = np.zeros((Nt * Nz, Nt * Nz), np.complex128)
    for m in range(Nt):
        X[m * Nz:(m + 1) * Nz, m * Nz:(m + 1) * Nz] = np.diag(n2_slice[m] - 1.0) + s * Dz
    Y = c * np.kron(Dt, np.eye(Nz))
    return X, Y


def dense_step(u, n2_slice, grid, rstar, dr=None, taylor=False):
    """u^{j+1} = solve([1+(1/4-d/4)X][1-(d/4)Y], [1+(1/4+d/4)X][1+(d/4)Y] u^j) (Eq. 4),
    or with the Taylor form of Eq. 3, T = X/2 - X^2/8:
    solve([1-(d/2)T][1-(d/4)Y], [1+(d/2)T][1+(d/4)Y] u^j)."""
    dr = grid.dr if dr is None else dr
    d = 1j * grid.k0 * dr
    X, Y = dense_operators(n2_slice, grid, rstar)
    Id = np.eye(X.shape[0])
    if taylor:
        T = X / 2 - (X @ X) / 8
        lhs = (Id - (d / 2) * T) @ (Id - (d / 4) * Y)
        rhs = (Id + (d / 2) * T) @ (Id + (d / 4) * Y)
    else:
        lhs = (Id + (0.25 - d / 4) * X) @ (Id - (d / 4) * Y)
        rhs = (Id + (0.25 + d / 4) * X) @ (Id + (d / 4) * Y)
    return np.linalg.solve(lhs, rhs @ u.ravel()).reshape(u.shape)


def active_slice(slice_r, r):
    k = 0
    for i, R in enumerate(slice_r):
        if R <= r:
            k = i
    return k


def y_range(g, j, y_midpoint):
    """Range at which Y is evaluated in step j: r_{j+1}, or the midpoint."""
    return g.r0 + (j + 0.5) * g.dr if y_midpoint else g.r0 + (j + 1) * g.dr


def check_dense(lib, periodic: bool, seed: int = 3, y_midpoint: bool = False, taylor: bool = False) -> float:
    wl = workloads.random_case(6, 5, periodic=periodic, K=3, steps=5, seed=seed, stride=1)
    g = wl.grid
    got = lib.march(g, wl.n2, wl.slice_r, wl.u0, y_midpoint=y_midpoint, taylor=taylor)
    u = wl.u0.copy()
    err = 0.0
    for j in range(g.steps):
        rstar = g.r0 + (j + 1) * g.dr
        u = dense_step(u, wl.n2[active_slice(wl.slice_r, rstar)], g, y_range(g, j, y_midpoint), taylor=taylor)
        err = max(err, relerr(got[j], u))
    return err


def check_interp_linear(lib, periodic: bool, y_midpoint: bool = False) -> float:
    """Range-interpolated medium.  The slices sample n^2(r) = A + B (r - r0), so
    the linear interpolation between them is that medium itself at every step
    range inside their span, and the first (last) slice before (after) it.  The
    interpolating march must equal dense Eq. 4 steps on those media; the steps
    cover both sides of the span and two intervals inside it."""
    wl = workloads.range_linear_case(6, 5, periodic=periodic, steps=9, seed=21)
    g = wl.grid
    A, B, R = wl.meta["A"], wl.meta["B"], wl.slice_r
    got = lib.march(g, wl.n2, R, wl.u0, interp=True, y_midpoint=y_midpoint)
    u = wl.u0.copy()
    err = 0.0
    for j in range(g.steps):
        r = g.r0 + (j + 1) * g.dr
        if r < R[0]:
            n2j = wl.n2[0]
        elif r >= R[-1]:
            n2j = wl.n2[-1]
        else:
            n2j = A + B * (r - g.r0)
        u = dense_step(u, n2j, g, y_range(g, j, y_midpoint))
        err = max(err, relerr(got[j], u))
    return err


# --------------------------------------------------------------------------
# closed-form discrete eigenmodes (homogeneous, theta-independent, real n0^2)
# --------------------------------------------------------------------------

def check_eigenmodes(lib, periodic: bool, n0sq: float, q: int = 2, p: int = 1,
                     steps: int = 7, y_midpoint: bool = False, taylor: bool = False) -> float:
    Nz, Nt = 9, 8
    g = workloads.Grid(Nz=Nz, Ntheta=Nt, dz=3.0, dtheta=(2 * math.pi / Nt) if periodic else 0.05,
                       dr=7.0, k0=0.3, r0=40.0, steps=steps, stride=steps, periodic=periodic)
    l = np.arange(Nz)
    m = np.arange(Nt)
    zmode = np.sin((q + 1) * math.pi * (l + 1) / (Nz + 1))
    if periodic:
        tmode = np.exp(2j * math.pi * p * m / Nt)
        mu_unit = -4.0 * math.sin(math.pi * p / Nt) ** 2
    else:
        tmode = np.sin((p + 1) * math.pi * (m + 1) / (Nt + 1))
        mu_unit = -4.0 * math.sin((p + 1) * math.pi / (2 * (Nt + 1))) ** 2
    u0 = (tmode[:, None] * zmode[None, :]).astype(np.complex128)
    n2 = np.full((1, Nt, Nz), n0sq, np.complex128)
    got = lib.march(g, n2, np.array([g.r0]), u0, y_midpoint=y_midpoint, taylor=taylor)[-1]
    d = 1j * g.k0 * g.dr
    s = 1.0 / (g.k0 * g.dz) ** 2
    lam = (n0sq - 1.0) - 4.0 * s * math.sin((q + 1) * math.pi / (2 * (Nz + 1))) ** 2
    alpha, beta = 0.25 - d / 4, 0.25 + d / 4
    gain = 1.0 + 0j
    for j in range(steps):
        c = 1.0 / (g.k0 * y_range(g, j, y_midpoint) * g.dtheta) ** 2
        mu = c * mu_unit
        if taylor:     # X's eigenvalue lam gives T = lam/2 - lam^2/8
            tl = lam / 2 - lam * lam / 8
            gain *= (1 + d / 2 * tl) / (1 - d / 2 * tl) * (1 + d / 4 * mu) / (1 - d / 4 * mu)
        else:
            gain *= (1 + beta * lam) / (1 + alpha * lam) * (1 + d / 4 * mu) / (1 - d / 4 * mu)
    return relerr(got, gain * u0)


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------

def check_norm_conservation(lib, periodic: bool, steps: int = 40, taylor: bool = False) -> float:
    """Real, theta-independent n^2 (depth- and range-dependent): X and Y commute
    and both factors are Cayley transforms, so ||u|| is conserved exactly."""
    rng = np.random.default_rng(11)
    Nz, Nt, K = 13, 7, 4
    wl = workloads.random_case(Nz, Nt, periodic=periodic, K=K, steps=steps, seed=11,
                               lossy=False, theta_dependent=False, stride=1)
    got = lib.march(wl.grid, wl.n2, wl.slice_r, wl.u0, taylor=taylor)
    n0 = np.linalg.norm(wl.u0)
    worst = 0.0
    for j in range(steps):
        drift = abs(np.linalg.norm(got[j]) - n0) / n0
        worst = max(worst, drift / (j + 1))      # allowed growth: ~1e-13 per step
    del rng
    return worst


def check_reversibility(lib, periodic: bool) -> float:
    """A step with +dr then a step with -dr at the same r* is the identity, for any
    medium (lossy, theta-dependent): S(-d) S(d) = B'^-1 A'^-1 A B B^-1 A^-1 A' B' = I."""
    wl = workloads.random_case(11, 6, periodic=periodic, K=1, steps=1, seed=5)
    g = wl.grid
    rstar = 150.0
    kw = dict(dz=g.dz, dtheta=g.dtheta, k0=g.k0, rstar=rstar, periodic=periodic)
    fwd = lib.step(wl.u0, wl.n2[0], dr=g.dr, **kw)
    back = lib.step(fwd, wl.n2[0], dr=-g.dr, **kw)
    return relerr(back, wl.u0)


def check_mirror(lib) -> float:
    """Walled sector with a mirror-symmetric medium and starter stays symmetric."""
    wl = workloads.random_case(10, 7, periodic=False, K=2, steps=6, seed=8, stride=6)
    n2 = 0.5 * (wl.n2 + wl.n2[:, ::-1, :])
    u0 = 0.5 * (wl.u0 + wl.u0[::-1, :])
    got = lib.march(wl.grid, n2, wl.slice_r, u0)[-1]
    return relerr(got[::-1, :], got)


def check_theta_uniform(lib) -> float:
    """Periodic, theta-independent medium and uniform starter: Yu = 0, every column
    equals the Ntheta = 1 march."""
    wl = workloads.random_case(12, 6, periodic=True, K=2, steps=6, seed=9, theta_dependent=False,
                               stride=3)
    col = wl.u0[0]
    u0 = np.broadcast_to(col, wl.u0.shape).copy()
    got = lib.march(wl.grid, wl.n2, wl.slice_r, u0)
    g1 = workloads.Grid(**{**wl.grid.__dict__, "Ntheta": 1})
    one = lib.march(g1, wl.n2[:, :1, :], wl.slice_r, col[None, :])
    return relerr(got, np.broadcast_to(one, got.shape))


# --------------------------------------------------------------------------
# the solvers alone
# --------------------------------------------------------------------------

def check_tridiag(lib, seed: int = 1) -> float:
    rng = np.random.default_rng(seed)
    worst = 0.0
    for n in (1, 2, 3, 5, 17, 64):
        for weak in (False, True):
            sub = rng.normal(size=n) + 1j * rng.normal(size=n)
            sup = rng.normal(size=n) + 1j * rng.normal(size=n)
            diag = rng.normal(size=n) + 1j * rng.normal(size=n)
            if weak:               # tiny diagonal: elimination must interchange rows
                diag *= 1e-3
            b = rng.normal(size=n) + 1j * rng.normal(size=n)
            A = np.diag(diag) + np.diag(sub[1:], -1) + np.diag(sup[:-1], 1)
            worst = max(worst, relerr(lib.tridiag_solve(sub, diag, sup, b), np.linalg.solve(A, b)))
    return worst


def check_penta(lib, seed: int = 6) -> float:
    """The banded (kl = ku = 2) elimination against LAPACK, including systems
    whose small diagonal forces row interchanges."""
    rng = np.random.default_rng(seed)
    worst = 0.0
    for n in (1, 2, 3, 4, 7, 40):
        for weak in (False, True):
            bands = rng.normal(size=(n, 5)) + 1j * rng.normal(size=(n, 5))
            if weak:
                bands[:, 2] *= 1e-3
            A = np.zeros((n, n), np.complex128)
            for i in range(n):
                for q in range(5):
                    c = i - 2 + q
                    if 0 <= c < n:
                        A[i, c] = bands[i, q]
            b = rng.normal(size=n) + 1j * rng.normal(size=n)
            worst = max(worst, relerr(lib.penta_solve(bands, b), np.linalg.solve(A, b)))
    return worst


def check_cyclic_fft(lib, seed: int = 2) -> float:
    """Constant-coefficient cyclic system = circulant: x = ifft(fft(b) / eig),
    eig_p = d + 2 e cos(2 pi p / n)."""
    rng = np.random.default_rng(seed)
    worst = 0.0
    for n in (3, 4, 8, 33, 256):
        dc = 1.0 + 3.0j
        e = -1.4j
        b = rng.normal(size=n) + 1j * rng.normal(size=n)
        eig = dc + 2 * e * np.cos(2 * math.pi * np.arange(n) / n)
        ref = np.fft.ifft(np.fft.fft(b) / eig)
        got = lib.cyclic_solve(np.full(n, e), np.full(n, dc), np.full(n, e), b)
        worst = max(worst, relerr(got, ref))
    return worst


def check_cyclic_dense(lib, seed: int = 4) -> float:
    """General (non-constant) cyclic tridiagonal against a dense LAPACK solve."""
    rng = np.random.default_rng(seed)
    worst = 0.0
    for n in (1, 2, 3, 6, 21):
        sub = rng.normal(size=n) + 1j * rng.normal(size=n)
        sup = rng.normal(size=n) + 1j * rng.normal(size=n)
        diag = 4.0 + rng.normal(size=n) + 1j * rng.normal(size=n)
        b = rng.normal(size=n) + 1j * rng.normal(size=n)
        A = np.zeros((n, n), np.complex128)
        for i in range(n):
            A[i, (i - 1) % n] += sub[i]
            A[i, i] += diag[i]
            A[i, (i + 1) % n] += sup[i]
        worst = max(worst, relerr(lib.cyclic_solve(sub, diag, sup, b), np.linalg.solve(A, b)))
    return worst


ALL_CHECKS = {
    "dense_walled": lambda L: check_dense(L, periodic=False),
    "dense_periodic": lambda L: check_dense(L, periodic=True),
    "eig_walled_1": lambda L: check_eigenmodes(L, False, 1.0),
    "eig_walled_09": lambda L: check_eigenmodes(L, False, 0.9),
    "eig_periodic_1": lambda L: check_eigenmodes(L, True, 1.0),
    "eig_periodic_09": lambda L: check_eigenmodes(L, True, 0.9),
    # the centred variant: Y at the step's midpoint r_j + dr/2
    "dense_walled_mid": lambda L: check_dense(L, periodic=False, y_midpoint=True),
    "dense_periodic_mid": lambda L: check_dense(L, periodic=True, y_midpoint=True),
    "eig_walled_mid": lambda L: check_eigenmodes(L, False, 0.9, y_midpoint=True),
    "eig_periodic_mid": lambda L: check_eigenmodes(L, True, 0.9, y_midpoint=True),
    # n^2 interpolated linearly in range
    "interp_walled": lambda L: check_interp_linear(L, periodic=False),
    "interp_periodic": lambda L: check_interp_linear(L, periodic=True),
    "interp_walled_mid": lambda L: check_interp_linear(L, periodic=False, y_midpoint=True),
    # the Taylor form of Eq. 3
    "dense_walled_taylor": lambda L: check_dense(L, periodic=False, taylor=True),
    "dense_periodic_taylor": lambda L: check_dense(L, periodic=True, taylor=True),
    "eig_walled_taylor": lambda L: check_eigenmodes(L, False, 0.9, taylor=True),
    "eig_periodic_taylor": lambda L: check_eigenmodes(L, True, 0.9, taylor=True),
    "norm_walled_taylor": lambda L: check_norm_conservation(L, False, taylor=True),
    "penta": check_penta,
    "norm_walled": lambda L: check_norm_conservation(L, False),
    "norm_periodic": lambda L: check_norm_conservation(L, True),
    "reverse_walled": lambda L: check_reversibility(L, False),
    "reverse_periodic": lambda L: check_reversibility(L, True),
    "mirror": check_mirror,
    "theta_uniform": check_theta_uniform,
    "tridiag": check_tridiag,
    "cyclic_fft": check_cyclic_fft,
    "cyclic_dense": check_cyclic_dense,
}

# per-check tolerance: 1e-12 relative, the norm drift is per step (1e-13 j)
TOLS = {k: TOL for k in ALL_CHECKS}
TOLS["norm_walled"] = 1e-13
TOLS["norm_periodic"] = 1e-13
TOLS["norm_walled_taylor"] = 1e-13
TOLS["penta"] = 1e-10         # weak-diagonal systems have condition numbers near 1e3

"""The FP64 oracle against what the mathematics fixes (CPU only).

Pins (paper Eq. 4-8, Fig. 2):
  * dense LU of the printed Eq. 4 on tiny grids, both boundaries, lossy and
    theta-dependent media, range-dependent slices (brute force);
  * closed-form per-step multipliers of the discrete sine/Fourier eigenmodes
    in a homogeneous theta-independent medium (pins the X and Y definitions,
    the sign of delta and the range r* at which operators are evaluated),
    both at r_{j+1} (Fig. 2) and in the centred variant with Y at r_j + dr/2;
  * exact norm conservation for real theta-independent media;
  * reversibility S(-delta) S(delta) = I for any medium;
  * mirror symmetry and the theta-uniform reduction to an Ntheta = 1 march;
  * the tridiagonal solver against LAPACK, the cyclic Sherman-Morrison solver
    against the circulant FFT solution and against LAPACK;
  * linearity and resume (march(2N) = march(N) followed by march(N)).
"""
import numpy as np
import pytest

import pins
import workloads


@pytest.mark.parametrize("name", sorted(pins.ALL_CHECKS))
def test_pin(oracle_lib, name):
    err = pins.ALL_CHECKS[name](oracle_lib)
    assert err < pins.TOLS[name], f"{name}: {err:.3e}"


def test_linearity(oracle_lib):
    wl = workloads.random_case(9, 6, periodic=False, K=2, steps=4, seed=21, stride=2)
    rng = np.random.default_rng(22)
    v0 = rng.normal(size=wl.u0.shape) + 1j * rng.normal(size=wl.u0.shape)
    a, b = 0.7 - 0.2j, -1.3 + 0.5j
    f = lambda u: oracle_lib.march(wl.grid, wl.n2, wl.slice_r, u)
    assert pins.relerr(f(a * wl.u0 + b * v0), a * f(wl.u0) + b * f(v0)) < 1e-12


@pytest.mark.parametrize("periodic", [False, True])
def test_resume(oracle_lib, periodic):
    wl = workloads.random_case(8, 6, periodic=periodic, K=3, steps=8, seed=23, stride=4)
    g = wl.grid
    full = oracle_lib.march(g, wl.n2, wl.slice_r, wl.u0)
    half = oracle_lib.march(g, wl.n2, wl.slice_r, wl.u0, steps=4, stride=4)
    rest = oracle_lib.march(g, wl.n2, wl.slice_r, half[-1], steps=4, stride=4, r0=g.r0 + 4 * g.dr)
    # identical arithmetic in identical order: bitwise equal
    assert np.array_equal(full[-1], rest[-1])


def test_lossy_norm_decreases(oracle_lib):
    """With Im(n^2) > 0 the field is damped (delta = +i k0 dr): the norm never grows."""
    wl = workloads.random_case(10, 6, periodic=True, K=1, steps=10, seed=31, lossy=True,
                               theta_dependent=False, stride=1)
    got = oracle_lib.march(wl.grid, wl.n2, wl.slice_r, wl.u0)
    norms = [np.linalg.norm(wl.u0)] + [np.linalg.norm(x) for x in got]
    assert all(b <= a * (1 + 1e-14) for a, b in zip(norms, norms[1:]))
    assert norms[-1] < norms[0] * 0.999


def test_empty_march(oracle_lib):
    wl = workloads.random_case(4, 3, periodic=False, steps=0)
    out = oracle_lib.march(wl.grid, wl.n2, wl.slice_r, wl.u0, steps=0, stride=1)
    assert out.shape == (0, 3, 4)


def test_single_point_grids(oracle_lib):
    """Nz = 1 and Ntheta = 1 (walled) reduce to scalar recurrences with closed forms."""
    g = workloads.Grid(Nz=1, Ntheta=1, dz=2.0, dtheta=0.1, dr=3.0, k0=0.5, r0=50.0,
                       steps=3, stride=3, periodic=False)
    n0 = 0.95 + 0.01j
    out = oracle_lib.march(g, np.full((1, 1, 1), n0), np.array([50.0]), np.ones((1, 1)))[-1]
    d = 1j * g.k0 * g.dr
    s = 1.0 / (g.k0 * g.dz) ** 2
    lam = (n0 - 1) - 2 * s
    gain = 1.0 + 0j
    for j in range(3):
        c = 1.0 / (g.k0 * (g.r0 + (j + 1) * g.dr) * g.dtheta) ** 2
        mu = -2 * c
        gain *= (1 + (0.25 + d / 4) * lam) / (1 + (0.25 - d / 4) * lam) * (1 + d / 4 * mu) / (1 - d / 4 * mu)
    assert abs(out[0, 0] - gain) < 1e-13

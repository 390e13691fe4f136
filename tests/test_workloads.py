"""Input recipes (CPU): the starters and the range-linear and broadband media."""
import math

import numpy as np

import workloads


def _grid(k0=0.3, Nz=64, dz=1.0):
    return workloads.Grid(Nz=Nz, Ntheta=5, dz=dz, dtheta=0.01, dr=1.0, k0=k0, r0=10.0, steps=1, stride=1,
                          periodic=False)


def test_image_starter_vanishes_at_the_surface():
    g = _grid()
    z = np.concatenate([[0.0], g.z])
    zs = 5.0
    plain = workloads.gaussian_starter(g, zs=zs)[2]
    img = workloads.gaussian_starter(g, zs=zs, image=True)[2]
    # the image term is the plain Gaussian mirrored about z = 0
    mirror = math.sqrt(g.k0) * np.exp(-(g.k0 ** 2) * (g.z + zs) ** 2 / 2) * plain[0] / (
        math.sqrt(g.k0) * math.exp(-(g.k0 ** 2) * (g.z[0] - zs) ** 2 / 2))
    assert np.allclose(plain - img, mirror, rtol=1e-12, atol=1e-15)
    # extended to z = 0 the imaged profile is zero there, and odd about it
    f = lambda zz: np.exp(-(g.k0 ** 2) * (zz - zs) ** 2 / 2) - np.exp(-(g.k0 ** 2) * (zz + zs) ** 2 / 2)
    assert abs(f(z[0])) == 0.0
    assert np.allclose(f(-g.z), -f(g.z), atol=1e-15)
    # deep below the source the image term is negligible
    assert abs(img[-1] - plain[-1]) < 1e-12 * abs(plain).max()


def test_range_linear_case_samples_a_linear_medium():
    wl = workloads.range_linear_case(8, 3, periodic=False, seed=4)
    A, B = wl.meta["A"], wl.meta["B"]
    for k, r in enumerate(wl.slice_r):
        assert np.allclose(wl.n2[k], A + B * (r - wl.grid.r0), rtol=0, atol=1e-15)
    assert np.all(np.diff(wl.slice_r) > 0)


def test_broadband_members_share_one_grid():
    bb = workloads.broadband(F=8, Nz=96, Ntheta=24, steps=40, T=256)
    g0 = bb.members[0].grid
    for wl, f in zip(bb.members, bb.freqs):
        g = wl.grid
        assert (g.Nz, g.Ntheta, g.dz, g.dtheta, g.dr, g.steps) == (g0.Nz, g0.Ntheta, g0.dz, g0.dtheta, g0.dr, g0.steps)
        assert math.isclose(g.k0, 2 * math.pi * f / workloads.C0)
        assert wl.n2 is bb.members[0].n2
    assert 1.0 / bb.dt > 2 * bb.freqs[-1]                  # the series is sampled above Nyquist
    assert abs(bb.W[0]) < 1e-20 and abs(bb.W[-1]) < 1e-20   # Hann window over the band
    assert math.isclose(g0.dz, workloads.C0 / bb.freqs[-1] / 8)

"""Pins of the oracle's pressure and transmission-loss output (CPU).

The paper recovers the pressure from the marched envelope as p = u w(r), with
w the Hankel function H0^(1)(k0 r) (Sec. 2; Fig. 2), and writes the
transmission loss -20 log10 |p| (Fig. 2; Fig. 5).  The oracle calls
scipy's hankel1 for H0^(1); these tests fix that call to things other than
itself:
  * Hankel's large-argument expansion of H0^(1) (DLMF 10.17.5), written out
    here with its coefficients a_k(0) = (-1)^k ((2k-1)!!)^2 / (k! 8^k), which
    pins the kind (1, not 2: the sign of the phase), the order (0) and the
    argument;
  * the tabulated first zeros of J0 and Y0 (Abramowitz & Stegun, Table 9.5),
    where H0^(1) is purely imaginary and purely real;
  * for a unit envelope, TL = -20 log10 |H0^(1)(k0 r)|, which approaches
    cylindrical spreading 10 log10(pi k0 r / 2) at long range;
  * the snapshot ranges r0 + (j+1) dr after step j.
"""
import math

import numpy as np
import pytest

import oracle


def _hankel_expansion(x, terms=8):
    """H0^(1)(x) ~ sqrt(2/(pi x)) e^{i(x - pi/4)} sum_k i^k a_k(0) / x^k."""
    s = np.zeros_like(x, dtype=np.complex128)
    a = 1.0
    for k in range(terms):
        if k > 0:
            a *= -((2 * k - 1) ** 2) / (8.0 * k)     # a_k(0) from a_{k-1}(0)
        s = s + (1j ** k) * a / x ** k
    return np.sqrt(2.0 / (np.pi * x)) * np.exp(1j * (x - np.pi / 4.0)) * s


def test_hankel_matches_large_argument_expansion():
    x = np.array([20.0, 41.888, 100.0, 837.76, 5000.0])
    h = oracle.hankel0(x)
    ref = _hankel_expansion(x)
    # the truncated asymptotic series is accurate to ~ a_8 / x^8 relative
    assert np.max(np.abs(h - ref) / np.abs(ref)) < 1e-9
    # the second kind (wrong sign of the phase) is far off
    assert np.max(np.abs(np.conj(h) - ref) / np.abs(ref)) > 0.5


def test_hankel_at_tabulated_bessel_zeros():
    j01 = 2.404825557695773      # first zero of J0
    y01 = 0.8935769662791675     # first zero of Y0
    h = oracle.hankel0(np.array([j01, y01]))
    assert abs(h[0].real) < 1e-14 and abs(h[0].imag) > 0.5
    assert abs(h[1].imag) < 1e-14 and abs(h[1].real) > 0.5


def test_transmission_loss_of_unit_field_is_cylindrical_spreading():
    k0 = 2 * math.pi * 100.0 / 1500.0
    r = np.array([100.0, 1000.0, 10000.0])
    u = np.ones((3, 2, 2), np.complex128)
    tl = oracle.transmission_loss(oracle.pressure(u, r, k0))
    x = k0 * r
    spread = 10.0 * np.log10(np.pi * x / 2.0)
    # J0^2 + Y0^2 = 2/(pi x) (1 - 1/(8 x^2) + 27/(128 x^4) - ...) (DLMF 10.18.17 with nu = 0), so
    # TL - spread = (10 / ln 10) / (8 x^2) + O(x^-4): within 1e-6 dB at x >= 40
    second = 10.0 / math.log(10.0) / (8.0 * x ** 2)
    assert np.max(np.abs(tl - spread[:, None, None] - second[:, None, None])) < 1e-6
    assert np.all(np.diff(tl[:, 0, 0]) > 0)            # loss grows with range


def test_transmission_loss_definition():
    p = np.array([1.0, 10.0, 1e-3, 3 + 4j], np.complex128)
    assert np.allclose(oracle.transmission_loss(p), [0.0, -20.0, 60.0, -20.0 * math.log10(5.0)], atol=1e-12)


def test_snapshot_ranges():
    r = oracle.snapshot_ranges(100.0, 5.0, steps=20, stride=7)
    assert np.allclose(r, [100.0 + 5.0 * 7, 100.0 + 5.0 * 14])
    assert oracle.snapshot_ranges(100.0, 5.0, steps=3, stride=4).size == 0


@pytest.mark.parametrize("mutant", ["kind2", "order1", "no_k0"])
def test_plausible_mistakes_fail_a_pin(mutant):
    """A wrong kind, order or argument in the Hankel factor breaks the pins."""
    from scipy.special import hankel1, hankel2
    x = np.array([20.0, 100.0, 837.76])
    wrong = {"kind2": hankel2(0, x), "order1": hankel1(1, x), "no_k0": hankel1(0, x / 0.41888)}[mutant]
    ref = _hankel_expansion(x)
    assert np.max(np.abs(wrong - ref) / np.abs(ref)) > 1e-3

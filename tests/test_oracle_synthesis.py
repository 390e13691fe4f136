"""Pins of the oracle's broadband synthesis (CPU).

s[r](t) = Re sum_i W_i p_i[r] e^{-2 pi i f_i t} is fixed here by things other
than its own formula:
  * one frequency: the cosine |W p| cos(2 pi f t - arg(W p));
  * a uniform frequency grid f_i = f0 + i df sampled at t_k = k / (F df):
    e^{-2 pi i f0 t_k} times the discrete Fourier transform over i of W_i p_i,
    numpy.fft.fft (the sign of the exponent and the sum over i);
  * the delay theorem: W_i e^{2 pi i f_i tau} gives s(t - tau).
"""
import math

import numpy as np
import pytest

import oracle


def _rand(rng, *shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


def test_single_frequency_is_a_cosine():
    rng = np.random.default_rng(1)
    p = _rand(rng, 1, 7)
    W = np.array([0.3 - 1.1j])
    f, t0, dt, T = 47.25, 3.1, 0.0037, 300
    s = oracle.synthesize([f], W, p, t0, dt, T)
    t = t0 + dt * np.arange(T)
    a = W[0] * p[0]
    ref = np.abs(a)[:, None] * np.cos(2 * math.pi * f * t[None, :] - np.angle(a)[:, None])
    assert np.max(np.abs(s - ref)) < 1e-12 * np.max(np.abs(a))


def test_uniform_grid_is_the_fft():
    rng = np.random.default_rng(2)
    F, R = 64, 5
    f0, df = 40.0, 0.25
    freqs = f0 + df * np.arange(F)
    W = _rand(rng, F)
    p = _rand(rng, F, R)
    T = F
    dt = 1.0 / (F * df)
    s = oracle.synthesize(freqs, W, p, 0.0, dt, T)
    t = dt * np.arange(T)
    ref = (np.exp(-2j * math.pi * f0 * t)[None, :] * np.fft.fft(W[:, None] * p, axis=0).T).real
    assert np.max(np.abs(s - ref)) < 1e-10 * np.max(np.abs(ref))


def test_delay_theorem():
    rng = np.random.default_rng(3)
    F, R, T = 20, 4, 50
    freqs = 30.0 + 1.7 * np.arange(F)
    W = _rand(rng, F)
    p = _rand(rng, F, R)
    tau, t0, dt = 0.137, 1.0, 0.004
    shifted = oracle.synthesize(freqs, W * np.exp(2j * math.pi * freqs * tau), p, t0, dt, T)
    direct = oracle.synthesize(freqs, W, p, t0 - tau, dt, T)
    assert np.max(np.abs(shifted - direct)) < 1e-10 * np.max(np.abs(direct))


@pytest.mark.parametrize("mutant", ["conj_phase", "imag_part", "no_weight", "t_without_t0"])
def test_plausible_mistakes_fail_a_pin(mutant):
    """Each planted mistake in a copy of the synthesis breaks the FFT pin."""
    rng = np.random.default_rng(4)
    F, R = 16, 3
    f0, df = 40.0, 0.5
    freqs = f0 + df * np.arange(F)
    W = _rand(rng, F)
    p = _rand(rng, F, R)
    dt = 1.0 / (F * df)
    t0 = 0.3 * dt

    def wrong(freqs, W, p, t0, dt, T):
        t = t0 + dt * np.arange(T)
        s = np.zeros((p.shape[1], T))
        for i in range(len(freqs)):
            w = 1.0 if mutant == "no_weight" else W[i]
            tt = dt * np.arange(T) if mutant == "t_without_t0" else t
            sign = +1 if mutant == "conj_phase" else -1
            z = w * p[i][:, None] * np.exp(sign * 2j * np.pi * freqs[i] * tt[None, :])
            s += z.imag if mutant == "imag_part" else z.real
        return s

    t = t0 + dt * np.arange(F)
    ref = (np.exp(-2j * math.pi * f0 * t)[None, :]
           * (np.fft.fft(W[:, None] * p * np.exp(-2j * math.pi * df * np.arange(F) * t0)[:, None], axis=0)).T).real
    assert np.max(np.abs(oracle.synthesize(freqs, W, p, t0, dt, F) - ref)) < 1e-10 * np.max(np.abs(ref))
    assert np.max(np.abs(wrong(freqs, W, p, t0, dt, F) - ref)) > 1e-3 * np.max(np.abs(ref))

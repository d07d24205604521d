"""Pins for the observed-data low-pass / resampling oracle (Blackman-windowed
sinc): what a band-limiting filter must do to sampled sinusoids, constants and
symmetric pulses, checked against closed forms (no second copy of the kernel).
"""
import numpy as np
import pytest


def _interior(t, W, T):
    return (t >= W) & (t <= T - W)


@pytest.mark.parametrize("dt_in,dt_out", [(1e-3, 1e-3), (6.25e-4, 2.1e-3), (2e-3, 1.3e-3)])
def test_passband_sinusoid_kept_with_exact_phase(orc, dt_in, dt_out):
    fc, W, T = 6.0, 0.6, 3.0
    nt_in, nt_out = int(T / dt_in) + 1, int(T / dt_out) + 1
    t_in = np.arange(nt_in) * dt_in
    t_out = np.arange(nt_out) * dt_out
    rng = np.random.default_rng(0)
    for f in (0.7, 1.9, 3.1):
        ph = rng.uniform(0, 2 * np.pi)
        x = np.sin(2 * np.pi * f * t_in + ph)[None, :, None]
        y = orc.lowpass(x, dt_in, nt_out, dt_out, fc, W)[0, :, 0]
        ref = np.sin(2 * np.pi * f * t_out + ph)   # zero phase: same sine at the new times
        k = _interior(t_out, W, T)
        assert np.max(np.abs(y[k] - ref[k])) < 2e-3, f


def test_stopband_sinusoid_removed(orc):
    fc, W, T, dt = 6.0, 0.6, 3.0, 5e-4
    t = np.arange(int(T / dt) + 1) * dt
    for f in (11.0, 17.0, 30.0):
        x = np.cos(2 * np.pi * f * t)[None, :, None]
        y = orc.lowpass(x, dt, len(t), dt, fc, W)[0, :, 0]
        assert np.max(np.abs(y[_interior(t, W, T)])) < 2e-3, f


def test_dc_gain_and_linearity(orc):
    fc, W, dt = 6.0, 0.5, 1e-3
    t = np.arange(2001) * dt
    y = orc.lowpass(np.ones((1, 2001, 2)), dt, 2001, dt, fc, W)
    k = _interior(t, W, t[-1])
    assert np.allclose(y[0, k], 1.0, atol=3e-4)   # Blackman pass-band ripple ~1.5e-4
    # zero beyond the record counts as zero: the edge value is about half
    assert 0.4 < y[0, 0, 0] < 0.6
    rng = np.random.default_rng(1)
    a, b = rng.normal(size=(2, 1, 300, 3))
    la = orc.lowpass(a, dt, 300, dt, fc, W)
    lb = orc.lowpass(b, dt, 300, dt, fc, W)
    assert np.allclose(orc.lowpass(2 * a - 3 * b, dt, 300, dt, fc, W), 2 * la - 3 * lb, atol=1e-12)


def test_symmetric_pulse_stays_symmetric_at_its_centre(orc):
    # a Ricker pulse centred at t0 filtered without resampling keeps its peak
    # time (zero phase) and its symmetry about t0
    fc, W, dt, f0 = 6.0, 0.6, 5e-4, 17.0
    t = np.arange(4001) * dt
    t0 = 1.0
    a = (np.pi * f0 * (t - t0)) ** 2
    x = ((1 - 2 * a) * np.exp(-a))[None, :, None]
    y = orc.lowpass(x, dt, len(t), dt, fc, W)[0, :, 0]
    c = int(round(t0 / dt))
    assert np.allclose(y[c - 1000:c], y[c + 1000:c:-1], atol=1e-12)
    assert np.argmax(np.abs(y)) == c
    # the 17 Hz Ricker keeps only its energy below ~6 Hz: much weaker
    assert np.max(np.abs(y)) < 0.1 * np.max(np.abs(x))

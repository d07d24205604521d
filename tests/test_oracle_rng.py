"""Pins for the oracle's counter-based random numbers.

Philox4x32-10 is checked against the known-answer vectors published with the
generator (Salmon et al., SC'11, Random123 distribution); the project-written
logarithm against Python's libm and the cosine against 200-bit\narithmetic; the normal deviates against
N(0, 1) by a Kolmogorov-Smirnov test.
"""
import math

import numpy as np
import pytest
from scipy import stats


@pytest.mark.parametrize("ctr,key,out", [
    ([0, 0, 0, 0], [0, 0], [0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8]),
    ([0xffffffff] * 4, [0xffffffff] * 2, [0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd]),
    ([0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344], [0xa4093822, 0x299f31d0],
     [0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1]),
])
def test_philox_known_answers(orc, ctr, key, out):
    assert list(orc.philox(ctr, key)) == out


def _ulps(a, b):
    return abs(a - b) / max(math.ulp(b), 1e-300)


def test_log_matches_libm(orc):
    rng = np.random.default_rng(0)
    us = np.concatenate([rng.uniform(0, 1, 20000), 2.0 ** -np.arange(1, 34),
                         [2.0 ** -33, 1 - 2.0 ** -33, 0.5, 0.70710678118654752, 0.7071067811865476]])
    worst = max(_ulps(orc.log(float(u)), math.log(u)) for u in us)
    assert worst <= 2.0


def test_cos2pi_matches_high_precision(orc):
    # reference in 200-bit arithmetic: libm's cos(2 * pi * t) itself carries
    # the rounding of its argument (~6e-16), the series must do better
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 200
    rng = np.random.default_rng(1)
    ts = np.concatenate([rng.uniform(0, 1, 4000), [2.0 ** -33, 0.125, 0.25, 0.375, 0.5,
                                                   0.625, 0.75, 0.875, 1 - 2.0 ** -33]])
    for t in ts:
        ref = float(mpmath.cos(2 * mpmath.pi * mpmath.mpf(float(t))))
        assert abs(orc.cos2pi(float(t)) - ref) <= 2.3e-16, t


def test_uniform_open_interval_and_moments(orc):
    u = np.array([orc.uniform(12795, 1, i, d, 2) for i in range(100) for d in range(50)])
    assert u.min() > 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01
    assert stats.kstest(u, "uniform").pvalue > 1e-3
    # distinct purposes give independent streams
    w = np.array([orc.uniform(12795, 1, i, d, 3) for i in range(100) for d in range(50)])
    assert abs(np.corrcoef(u, w)[0, 1]) < 0.05


def test_normal_is_standard(orc):
    z = np.array([orc.normal(7, 3, i, d) for i in range(200) for d in range(50)])
    assert abs(z.mean()) < 0.04
    assert abs(z.std() - 1.0) < 0.03
    assert stats.kstest(z, "norm").pvalue > 1e-3

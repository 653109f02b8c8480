"""Pins of the oracle's quintic kernel (§3, Eq. 18) against what the paper prints and calculus.

The paper prints the three normalisation constants of the kernel; each must make the printed
polynomial integrate to one in its own dimension.  That ties the oracle's polynomial (every piece
and coefficient) to the paper: a wrong coefficient breaks at least one of the three integrals.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "kernel_constants.json")))


def _poly(orc, b):
    """The oracle's W(b) with its 2D constant divided out (the bare piecewise polynomial)."""
    h = 0.37
    return orc.lib().orc_W(b, h) / orc.kernel_ad(h)


def _quad(f):
    tot = 0.0
    for a in range(3):  # integrate piece by piece: the kernel's breakpoints are b = 1, 2, 3
        v, _ = integrate.quad(f, a, a + 1, epsabs=1e-15, epsrel=1e-14, limit=200)
        tot += v
    return tot


def test_2d_constant_matches_paper(orc):
    g = GOLD["a_d_2d"]
    for h in (0.01, 1.3 / 64, 0.5):
        want = g["numerator"] / (g["denominator_over_pi"] * math.pi * h ** g["h_power"])
        assert orc.kernel_ad(h) == pytest.approx(want, rel=1e-15)


def test_printed_constants_normalise_the_polynomial(orc):
    # 2D: int W dA = a_d int P(b) 2 pi b h^2 db = 1 with a_d = 7/(478 pi h^2)
    g2 = GOLD["a_d_2d"]
    i2 = _quad(lambda b: _poly(orc, b) * 2.0 * math.pi * b)
    assert i2 * g2["numerator"] / (g2["denominator_over_pi"] * math.pi) == pytest.approx(1.0, abs=1e-12)
    # 3D: the printed 3/(359 pi h^3) normalises to 0.28 %; the exact constant of the printed
    # polynomial is 1/(120 pi h^3), since int_0^a (a-b)^5 b^2 db = a^8/168 and
    # (3^8 - 6*2^8 + 15)/168 = 30.  Only the 2D constant enters the method.
    g3 = GOLD["a_d_3d"]
    i3 = _quad(lambda b: _poly(orc, b) * 4.0 * math.pi * b * b)
    assert i3 == pytest.approx(120.0 * math.pi, rel=1e-12)
    assert i3 * g3["numerator"] / (g3["denominator_over_pi"] * math.pi) == pytest.approx(1.0, rel=3e-3)
    # 1D: the printed "120/h" only normalises as 1/(120 h)
    g1 = GOLD["a_d_1d_reading"]
    i1 = 2.0 * _quad(lambda b: _poly(orc, b))
    assert i1 * g1["numerator"] / g1["denominator"] == pytest.approx(1.0, abs=1e-12)
    assert i1 * 120.0 != pytest.approx(1.0, rel=0.5)


def test_2d_normalisation_in_physical_units(orc):
    h = 1.3 / 64
    f = lambda r: orc.lib().orc_W(r / h, h) * 2.0 * math.pi * r
    tot = sum(integrate.quad(f, a * h, (a + 1) * h, epsabs=1e-15, epsrel=1e-13)[0] for a in range(3))
    assert tot == pytest.approx(1.0, abs=1e-11)


def test_support_and_smoothness(orc):
    h = 0.2
    k = GOLD["support_kappa"]
    W = lambda b: orc.lib().orc_W(b, h)
    dW = lambda b: orc.lib().orc_dWdb(b, h)
    assert W(k) == 0.0 and dW(k) == 0.0
    assert W(k + 1e-9) == 0.0 and W(4.0) == 0.0
    ad = orc.kernel_ad(h)
    for bp in (1.0, 2.0):  # value and slope continuous across the breakpoints: a jump would be
        e = 1e-8           # of order a_d, the change across 2e is bounded by the next derivative
        assert abs(W(bp - e) - W(bp + e)) <= 3 * e * 100 * ad
        assert abs(dW(bp - e) - dW(bp + e)) <= 3 * e * 1000 * ad
    # (3-b)^5 vanishes to 4th order at the support edge
    assert W(3.0 - 1e-3) / W(3.0 - 2e-3) == pytest.approx((1e-3 / 2e-3) ** 5, rel=1e-9)


def test_derivative_matches_finite_differences(orc):
    h = 0.13
    W = lambda b: orc.lib().orc_W(b, h)
    for b in np.linspace(0.05, 2.95, 59):
        if abs(b - 1.0) < 1e-3 or abs(b - 2.0) < 1e-3:
            continue
        e = 1e-5
        fd = (W(b + e) - W(b - e)) / (2 * e)
        assert orc.lib().orc_dWdb(b, h) == pytest.approx(fd, rel=1e-7, abs=1e-9 * abs(W(0.0)))


def test_monotone_decreasing(orc):
    h = 1.0
    bs = np.linspace(0.0, 3.0, 301)
    w = orc.W(bs, h)
    assert np.all(np.diff(w) <= 0.0)
    assert np.all(orc.dWdb(bs[1:], h) <= 0.0)
    assert orc.lib().orc_dWdb(0.0, h) == pytest.approx(0.0, abs=1e-12)

"""Pins of the oracle's smoothing kernel (M4 cubic spline with support 2h).

The paper names the cubic spline (Section 2) but prints no formula; these
checks tie the oracle's W to properties any SPH kernel must have, independent
of how the oracle writes it: unit normalisation, the derivative relations, and
continuity at the spline knots.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore")


def test_normalisation_gauss_legendre(orc):
    # integral over R^3 of W(r, h) = 4 pi int_0^{2h} r^2 W dr = 1.  Gauss-Legendre
    # with 8 nodes is exact for the degree-5 polynomial on each spline piece.
    xg, wg = np.polynomial.legendre.leggauss(8)
    for h in (0.01, 0.3, 1.0, 7.5):
        total = 0.0
        for a, b in ((0.0, h), (h, 2.0 * h)):
            r = 0.5 * (b - a) * xg + 0.5 * (b + a)
            total += 0.5 * (b - a) * sum(wi * 4.0 * math.pi * ri * ri * orc.W(ri, h)
                                         for ri, wi in zip(r, wg))
        assert abs(total - 1.0) < 1e-14, (h, total)


def test_centre_value_and_support(orc):
    for h in (0.5, 2.0):
        assert orc.W(0.0, h) == pytest.approx(1.0 / (math.pi * h ** 3), rel=1e-15)
        assert orc.W(2.0 * h, h) == 0.0
        assert orc.W(2.5 * h, h) == 0.0
        assert orc.W(1.999999 * h, h) > 0.0


def test_knot_continuity(orc):
    eps = 1e-12
    for q in (1.0, 2.0):
        assert orc.w(q - eps) == pytest.approx(orc.w(q + eps), abs=1e-10)
        assert orc.dw(q - eps) == pytest.approx(orc.dw(q + eps), abs=1e-10)
    # w(1) = 1/4 and w'(1) = -3/4 (values of the M4 spline at its inner knot)
    assert orc.w(1.0) == pytest.approx(0.25, abs=1e-15)
    assert orc.dw(1.0) == pytest.approx(-0.75, abs=1e-15)


def test_dWdr_matches_finite_difference(orc):
    h = 0.7
    for r in np.linspace(0.05, 1.95, 23) * h:
        d = 1e-6 * h
        fd = (orc.W(r + d, h) - orc.W(r - d, h)) / (2 * d)
        assert orc.dWdr(r, h) == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_dWdh_matches_finite_difference(orc):
    h = 0.9
    for r in np.linspace(0.0, 1.95, 21) * h:
        d = 1e-6 * h
        fd = (orc.W(r, h + d) - orc.W(r, h - d)) / (2 * d)
        assert orc.dWdh(r, h) == pytest.approx(fd, rel=1e-6, abs=1e-9)


def test_kernel_is_monotone_decreasing(orc):
    q = np.linspace(0.0, 2.0, 401)
    vals = [orc.w(t) for t in q]
    assert all(a >= b for a, b in zip(vals, vals[1:]))

"""Pins of the oracle's kernel functions (Eqs. 22 and 23) against closed
forms, quadrature and finite differences."""
import math

import numpy as np
import pytest
from scipy import integrate

SIG = 5.0 / (14.0 * math.pi)


def _radial_integral(f, support):
    val, _ = integrate.quad(lambda r: 2.0 * math.pi * r * f(r), 0.0, support, points=[support / 2], limit=200,
                            epsabs=1e-14, epsrel=1e-13)
    return val


@pytest.mark.parametrize("h", [0.013, 0.0026, 1.0])
def test_cubic_normalised_with_reading_constant(orc, h):
    # Eq. 6: the normalised kernel integrates to 1 over the 2-D plane.
    assert _radial_integral(lambda r: orc.w_cubic(r, h, SIG), 2 * h) == pytest.approx(1.0, abs=1e-11)


def test_cubic_printed_constant_integrates_to_three(orc):
    # The constant printed in Eq. 22, 15/(14 pi), gives 3, so the normalised kernel takes 5/(14 pi).
    h = 0.7
    assert _radial_integral(lambda r: orc.w_cubic(r, h, 15.0 / (14.0 * math.pi)), 2 * h) == pytest.approx(3.0, abs=1e-10)


@pytest.mark.parametrize("h", [0.013, 1.0])
def test_spiky_normalised(orc, h):
    # Eq. 23 is normalised in 2-D (statement after Eq. 23).
    assert _radial_integral(lambda r: orc.w_spiky(r, h), h) == pytest.approx(1.0, abs=1e-11)


def test_cubic_closed_form_values(orc):
    h = 0.3
    c = SIG / h**2
    assert orc.w_cubic(0.0, h, SIG) == pytest.approx(4.0 * c, rel=1e-15)  # (2)^3 - 4 (1)^3
    assert orc.w_cubic(h, h, SIG) == pytest.approx(c, rel=1e-14)          # (2-1)^3
    assert orc.w_cubic(1.5 * h, h, SIG) == pytest.approx(c * 0.125, rel=1e-14)
    assert orc.w_cubic(2.0 * h, h, SIG) == 0.0
    assert orc.w_cubic(2.5 * h, h, SIG) == 0.0
    # continuity of W and dW/dr across q = 1 and q = 2
    e = 1e-9
    assert orc.w_cubic(h - e, h, SIG) == pytest.approx(orc.w_cubic(h + e, h, SIG), rel=1e-7)
    assert orc.dw_cubic(h - e, h, SIG) == pytest.approx(orc.dw_cubic(h + e, h, SIG), rel=1e-7)
    assert abs(orc.dw_cubic(2 * h - e, h, SIG)) < 1e-12
    assert orc.dw_cubic(0.0, h, SIG) == 0.0   # smooth at the centre


def test_spiky_closed_form_values(orc):
    h = 0.2
    assert orc.w_spiky(0.0, h) == pytest.approx(10.0 / (math.pi * h**2), rel=1e-14)
    assert orc.dw_spiky(0.0, h) == pytest.approx(-30.0 / (math.pi * h**3), rel=1e-14)  # non-vanishing at 0
    assert orc.w_spiky(h, h) == 0.0
    assert orc.w_spiky(1.1 * h, h) == 0.0


@pytest.mark.parametrize("q", [0.05, 0.3, 0.77, 1.2, 1.6, 1.95])
def test_derivatives_match_finite_differences(orc, q):
    h = 0.013
    r = q * h
    d = 1e-7 * h
    fd = (orc.w_cubic(r + d, h, SIG) - orc.w_cubic(r - d, h, SIG)) / (2 * d)
    assert orc.dw_cubic(r, h, SIG) == pytest.approx(fd, rel=1e-6, abs=1e-6 * abs(orc.dw_cubic(h, h, SIG)))
    if q < 1.0:
        fds = (orc.w_spiky(r + d, h) - orc.w_spiky(r - d, h)) / (2 * d)
        assert orc.dw_spiky(r, h) == pytest.approx(fds, rel=1e-6)

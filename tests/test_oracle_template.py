"""Pins of the transit template (quadratic limb darkening, central transit)."""

import math

import numpy as np
import pytest

from oracle import grid

U1, U2 = 0.4, 0.25
# mean of the continuous profile over the chord: 1 - u1 (1 - pi/4) - u2 (5/3 - pi/2)
LIMIT = 1.0 - U1 * (1.0 - math.pi / 4.0) - U2 * (5.0 / 3.0 - math.pi / 2.0)


def test_closed_form_limit_value():
    assert LIMIT == pytest.approx(0.8901917, abs=5e-8)


@pytest.mark.parametrize("d", [1, 3, 9, 101, 2001])
def test_centre_is_one_for_odd_d(d):
    s = grid.template(d, U1, U2)
    assert s[d // 2] == 1.0


@pytest.mark.parametrize("d", [2, 7, 64, 1000])
def test_symmetric_and_bounded(d):
    s = grid.template(d, U1, U2)
    assert np.allclose(s, s[::-1], rtol=0, atol=1e-13)   # symmetric up to rounding of x
    assert np.all(s > 0.0) and np.all(s <= 1.0)
    # monotone towards the centre
    h = s[: (d + 1) // 2]
    assert np.all(np.diff(h) >= 0)


def test_mean_converges_to_integral():
    # midpoint rule on a sqrt-type edge: error shrinks like D^(-3/2)
    errs = []
    for d in (10, 100, 1000, 10000):
        errs.append(abs(grid.template(d, U1, U2).mean() - LIMIT))
    assert errs[0] == pytest.approx(0.00601, abs=5e-5)
    for a, b in zip(errs, errs[1:]):
        assert 20.0 < a / b < 45.0        # 10^(3/2) = 31.6


def test_single_point_template():
    assert grid.template(1, U1, U2)[0] == 1.0


def test_uniform_disk_is_a_box():
    # no limb darkening: the template reduces to the BLS box
    assert np.all(grid.template(50, 0.0, 0.0) == 1.0)


def test_edge_value():
    # first midpoint of D points: x = 1/(2D), |2x - 1| = 1 - 1/D
    d = 40
    r = 1.0 - 1.0 / d
    mu = math.sqrt(1.0 - r * r)
    want = 1.0 - U1 * (1.0 - mu) - U2 * (1.0 - mu) ** 2
    assert grid.template(d, U1, U2)[0] == pytest.approx(want, rel=1e-15)

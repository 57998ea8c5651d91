"""Host diagnostics of an exported phase field, on shapes of known size: a disc of radius R
(every ray crosses at R, no orientation spread), a regular hexagon (tips at the circumradius,
the contour between arms at the inradius: notch ratio 1), linear growth (tip speed) and
uniform fields (area)."""
import math

import numpy as np
import pytest

from paper_2101_07163_gb300 import diagnostics as D

N, CX, CY = 160, 80.3, 79.6


def grid():
    y, x = np.mgrid[0:N, 0:N].astype(np.float64)
    return x - CX, y - CY


def disc(R, width=2.0):
    x, y = grid()
    return np.tanh((R - np.hypot(x, y)) / width)


def hexagon(Rc, width=2.0):
    # vertices along 0, 60, ... degrees; edge normals along 30, 90, ... degrees
    x, y = grid()
    d = np.max([x * math.cos(math.radians(30 + 60 * k)) + y * math.sin(math.radians(30 + 60 * k))
                for k in range(6)], axis=0)
    return np.tanh((Rc * math.sqrt(3) / 2 - d) / width)


@pytest.mark.parametrize("angle", [0.0, 17.0, 45.0, 60.0, 123.0, 270.0])
def test_rays_cross_a_disc_at_its_radius(angle):
    assert D.tip_radius(disc(31.7), CX, CY, angle) == pytest.approx(31.7, abs=0.02)


def test_disc_has_no_orientation_spread():
    tips = D.arm_tips(disc(25.2), CX, CY, fold=6)
    assert D.orientation_spread(tips) < 1e-3
    assert len(D.arm_tips(disc(25.2), CX, CY, fold=4)) == 4


def test_hexagon_tips_and_notch_ratio():
    # bilinear samples round a sharp vertex: near it the off-ray samples lie on the other face,
    # so the crossing reads up to 0.3 cells short of the circumradius; the faces are exact
    h = hexagon(40.0)
    tips = D.arm_tips(h, CX, CY, fold=6)
    assert np.all(np.abs(np.array(tips) - 40.0) < 0.35)
    assert D.tip_radius(h, CX, CY, 30.0) == pytest.approx(40.0 * math.sqrt(3) / 2, abs=0.02)
    assert D.notch_ratio(h, CX, CY) == pytest.approx(1.0, abs=1e-2)
    # a disc of the same circumradius bulges between the arms
    assert D.notch_ratio(disc(40.0), CX, CY) > 1.1


def test_rays_outside_the_crystal_or_the_grid_give_nan():
    assert math.isnan(D.tip_radius(disc(10.0), 5.0, 5.0, 0.0))      # starts in the vapour
    assert math.isnan(D.tip_radius(np.ones((N, N)), CX, CY, 0.0))    # never crosses


def test_tip_speed_and_area():
    t = np.arange(0, 100, 10.0)
    assert D.tip_speed(t, 3.0 + 0.25 * t) == pytest.approx(0.25, rel=1e-12)
    with pytest.raises(ValueError):
        D.tip_speed([1.0], [2.0])
    assert D.solid_area(np.ones((8, 5)), dx=0.4) == pytest.approx(40 * 0.16, rel=1e-15)
    assert D.solid_area(-np.ones((8, 5))) == 0.0

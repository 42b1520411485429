"""The circle-fit contact angle (Sec. 3.2) on synthetic menisci of known shape (no GPU).

phi is a tanh profile of width sqrt(2) across an exact circular arc that meets the two
wall planes (the boundary-node rows j = 0 and j = H - 1) at a chosen angle; the fit must
return that angle.
"""
import math

import numpy as np
import pytest

from paper_0911_0459_gb300 import meniscus


def synthetic(theta_deg, H=39, nx=300, x0=60, L=230, apex=80.0, jc=None, ny=None, ramp=False):
    ny = ny or H + 1
    jc = (H - 1) / 2.0 if jc is None else jc
    d = jc   # distance from the centre to the j = 0 wall (the test picks jc so both walls agree)
    c = math.cos(math.radians(theta_deg))
    phi = np.zeros((ny, nx))
    x = np.arange(nx, dtype=float)
    for j in range(H):
        if abs(c) < 1e-12:
            xa = x0 + apex
        else:
            R = d / abs(c)
            if c > 0:   # wetting: centre on the gas side, interface on the circle's left branch
                xc = x0 + apex + R
                xa = xc - math.sqrt(max(R * R - (j - jc) ** 2, 0.0))
            else:       # non-wetting: centre on the liquid side, right branch
                xc = x0 + apex - R
                xa = xc + math.sqrt(max(R * R - (j - jc) ** 2, 0.0))
        # ramp: a clipped linear profile, on which the interpolated crossing is exact
        phi[j] = np.clip(xa - x, -3.0, 3.0) if ramp else np.tanh((xa - x) / math.sqrt(2.0))
    return phi, (x0, L, 0, H)


@pytest.mark.parametrize("theta", [30.0, 45.0, 60.0, 63.0, 80.0, 100.0, 120.0])
def test_circle_fit_recovers_the_contact_angle(theta):
    phi, geom = synthetic(theta)
    assert abs(meniscus.contact_angle(phi, *geom) - theta) < 0.1


def test_flat_interface_is_ninety_degrees():
    phi, geom = synthetic(90.0)
    assert abs(meniscus.contact_angle(phi, *geom) - 90.0) < 1e-6


def test_band_that_wraps_in_y():
    """A band starting at row ny - 10 that continues through row 0 (periodic in y)."""
    phi, (x0, L, _, H) = synthetic(50.0, ny=60)
    shifted = np.roll(phi, 50, axis=0)     # band rows 0..38 -> 50..59, 0..28
    assert abs(meniscus.contact_angle(shifted, x0, L, 50, H) - 50.0) < 0.1


def test_circle_fit_is_exact_on_a_circle():
    t = np.linspace(-1.0, 1.0, 25)
    xc, yc, R = 3.5, -2.0, 17.0
    x, y = xc + R * np.cos(t), yc + R * np.sin(t)
    fx, fy, fR = meniscus.fit_circle(x, y)
    assert abs(fx - xc) < 1e-9 and abs(fy - yc) < 1e-9 and abs(fR - R) < 1e-9


@pytest.mark.parametrize("margin", [1, 4, 10])
def test_rows_left_out_next_to_the_walls_do_not_move_an_exact_arc(margin):
    """The wall planes stay at the boundary-node rows whatever the rows fitted: with
    exact interface points the fit of any subset of rows gives the angle exactly."""
    phi, geom = synthetic(63.0, ramp=True)
    assert abs(meniscus.contact_angle(phi, *geom, margin=margin) - 63.0) < 1e-6
    x, j = meniscus.interface_points(phi, *geom, margin=margin)
    assert j.min() == margin and j.max() == geom[3] - 1 - margin

"""Contact angle of a meniscus from the order-parameter field, as the paper measures it
(Sec. 3.2): a least-squares fit of the interface profile to a circular section.

The interface in the tube is taken row by row: in every fluid row of the tube's band
(band-local coordinate j = 0 .. H - 1), the first sign change of phi scanning from the
inlet, linearly interpolated.  The two boundary-node rows (j = 0 and j = H - 1) are
the wall planes, where the wetting condition is imposed; the rows strictly between
them are fitted.  The circle (centre (xc, jc), radius R) is the algebraic least-squares
fit x^2 + j^2 + D x + E j + F = 0.  At a wall plane at distance d from the centre, the
interface meets the wall at cos(theta) = s d / R, with s = +1 when the centre lies on
the gas side of the interface (a meniscus concave towards the gas, theta < 90) and
s = -1 otherwise; the angle returned is the mean over the two walls, in degrees, measured
through the liquid.  phi > 0 is the liquid.
"""
from __future__ import annotations

import math
from typing import Tuple

import numpy as np


def interface_points(phi: np.ndarray, tube_x0: int, tube_len: int, tube_y0: int, tube_h: int,
                     margin: int = 1) -> Tuple[np.ndarray, np.ndarray]:
    """(x, j) of the phi = 0 crossing in each band row margin .. H - 1 - margin that has
    one, with x measured from the tube inlet (x = 0 at column tube_x0)."""
    ny, nx = phi.shape
    xs, js = [], []
    cols = (tube_x0 + np.arange(tube_len)) % nx
    for j in range(margin, tube_h - margin):
        row = phi[(tube_y0 + j) % ny, cols]
        pos = row > 0
        # first liquid -> gas change scanning from the inlet
        k = np.nonzero(pos[:-1] & ~pos[1:])[0]
        if len(k) == 0:
            continue
        k = int(k[0])
        xs.append(k + row[k] / (row[k] - row[k + 1]))
        js.append(float(j))
    return np.array(xs), np.array(js)


def fit_circle(x: np.ndarray, y: np.ndarray) -> Tuple[float, float, float]:
    """Centre and radius of the algebraic least-squares circle through (x, y)."""
    A = np.stack([x, y, np.ones_like(x)], axis=1)
    b = -(x * x + y * y)
    (D, E, F), *_ = np.linalg.lstsq(A, b, rcond=None)
    xc, yc = -D / 2.0, -E / 2.0
    return float(xc), float(yc), float(math.sqrt(max(xc * xc + yc * yc - F, 0.0)))


def contact_angle(phi: np.ndarray, tube_x0: int, tube_len: int, tube_y0: int, tube_h: int,
                  margin: int = 1) -> float:
    """Contact angle in degrees from the circular fit of the interface rows margin ..
    H - 1 - margin (nan if fewer than three rows have an interface)."""
    x, j = interface_points(phi, tube_x0, tube_len, tube_y0, tube_h, margin)
    if len(x) < 3:
        return float("nan")
    if np.ptp(x) <= 1e-9 * max(1.0, float(np.abs(x).max())):
        return 90.0  # a straight interface across the tube (the circle degenerates)
    xc, jc, R = fit_circle(x, j)
    # centre on the gas side: beyond the interface in the filling direction
    s = 1.0 if xc > float(np.mean(x)) else -1.0
    thetas = []
    for d in (jc - 0.0, (tube_h - 1.0) - jc):
        thetas.append(math.degrees(math.acos(max(-1.0, min(1.0, s * d / R)))))
    return float(np.mean(thetas))


def lattice_contact_angle(lat) -> float:
    """contact_angle of a Lattice (binding) from its current fields."""
    _, _, _, phi = lat.fields()
    w = lat.walls
    return contact_angle(phi, w.tube_x0, w.tube_len, w.tube_y0, w.tube_h)

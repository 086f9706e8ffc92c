"""Oracle pin: the Taylor deformation D = (L - B)/(L + B) (Sec. 5.5).

A uniform ellipse with semi-axes a >= b has second moments a^2/4 and b^2/4
along its axes, so L and B (twice the semi-axes) give D = (a - b)/(a + b)
exactly.  The ellipse is rasterised onto the node lattice as the area fraction
of each cell (16 x 16 sub-samples), phi = 2 fraction - 1, at an off-lattice
centre and several orientations.  The lattice moments miss the 1/12 variance
of each cell, an error that falls as 1/R^2: the test asks for D within that
bound at two sizes and for the second-order trend between them.  Taking the
variance where its square root belongs would give (a^2 - b^2)/(a^2 + b^2)
(0.385 instead of 0.2 here), a wrong cross moment or discriminant would make
D depend on the orientation.
"""
import math

import numpy as np
import pytest


def _ellipse(n, a, b, theta, xc, yc, sub=16):
    """phi = 2 * (cell area fraction inside the ellipse) - 1 on an n x n grid of
    nodes at integer coordinates, the cell of node (x, y) being the unit square
    centred on it."""
    s = (np.arange(sub) + 0.5) / sub - 0.5
    X = (np.arange(n)[None, :, None, None] + s[None, None, None, :]) - xc
    Y = (np.arange(n)[:, None, None, None] + s[None, None, :, None]) - yc
    c, si = math.cos(theta), math.sin(theta)
    u = c * X + si * Y
    v = -si * X + c * Y
    inside = (u / a) ** 2 + (v / b) ** 2 <= 1.0
    frac = inside.mean(axis=(2, 3))
    return 2.0 * frac - 1.0


@pytest.mark.parametrize("theta", [0.0, 0.5, math.pi / 2, 2.2])
def test_taylor_D_of_uniform_ellipses(orc, theta):
    err = {}
    for a, b in ((12.0, 8.0), (24.0, 16.0)):
        n = int(2 * a + 12)
        phi = _ellipse(n, a, b, theta, n / 2 + 0.31, n / 2 - 0.17)
        D = orc.taylor_D({"phi": phi})
        err[a] = abs(D - (a - b) / (a + b))
    assert err[12.0] < 1.2e-3 and err[24.0] < 3e-4, err
    assert err[12.0] / err[24.0] > 3.0, err


def test_taylor_D_of_a_disc_is_zero_and_of_a_line_is_one(orc):
    phi = _ellipse(60, 20.0, 20.0, 0.0, 30.13, 29.71)
    assert orc.taylor_D({"phi": phi}) < 1e-3
    # all the fluid-1 weight on one row: B = 0, D = 1
    phi = -np.ones((20, 40))
    phi[7, 5:30] = 1.0
    assert orc.taylor_D({"phi": phi}) == pytest.approx(1.0, abs=1e-12)

"""Pins of the oracle's rising-bubble quantities (Sec. 5.4: Eqs. quantify-yc,
quantify-uc, circularity) against geometry that does not go through the
oracle's own formulas: clipped straight lines, circles and ellipses of known
perimeter, exact mirror symmetry, lattice-point counts and hand-worked
marching-squares cells."""
import math

import numpy as np
import pytest


def _grid(nx, ny):
    return np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))


def _clip_length(a, b, c, nx, ny):
    """Length of the line a x + b y + c = 0 inside [0, nx-1] x [0, ny-1]
    (Liang-Barsky clipping of the parametric line)."""
    # a point on the line and its direction
    if abs(b) > abs(a):
        p0 = np.array([0.0, -c / b])
    else:
        p0 = np.array([-c / a, 0.0])
    d = np.array([b, -a]) / math.hypot(a, b)
    lo, hi = -1e9, 1e9
    for k, (mn, mx) in enumerate(((0.0, nx - 1.0), (0.0, ny - 1.0))):
        if abs(d[k]) < 1e-15:
            if not (mn <= p0[k] <= mx):
                return 0.0
            continue
        t1, t2 = (mn - p0[k]) / d[k], (mx - p0[k]) / d[k]
        lo, hi = max(lo, min(t1, t2)), min(hi, max(t1, t2))
    return max(0.0, hi - lo)


@pytest.mark.parametrize("a,b,c", [(0.3, 1.0, -7.4), (1.0, 0.45, -11.2), (-0.8, 0.6, 2.3),
                                   (0.0, 1.0, -5.5)])
def test_linear_field_contour_is_the_clipped_line(orc, a, b, c):
    # marching squares interpolates linearly along edges: exact on a plane
    nx, ny = 23, 17
    x, y = _grid(nx, ny)
    phi = a * x + b * y + c
    got = orc.contour_length(phi, False, False)
    assert got == pytest.approx(_clip_length(a, b, c, nx, ny), rel=1e-12, abs=1e-12)


def test_horizontal_line_wraps_in_periodic_x(orc):
    nx, ny = 20, 11
    x, y = _grid(nx, ny)
    phi = y - 4.3
    assert orc.contour_length(phi, True, False) == pytest.approx(nx, rel=1e-14)
    assert orc.contour_length(phi, False, False) == pytest.approx(nx - 1, rel=1e-14)
    # wrapping in y joins y = ny - 1 (phi = 5.7) to y = 0 (phi = -4.3): the
    # ramp's jump is a second, horizontal contour
    assert orc.contour_length(phi, False, True) == pytest.approx(2 * (nx - 1), rel=1e-14)


def test_saddle_cells_by_the_centre_value(orc):
    # inside corners 0 and 2 of the cell (phi = -3), centre mean -1 < 0: the
    # inside corners connect, the two segments cut off the outside corners,
    # legs of 1/4 each: 2 * sqrt(2) / 4
    assert orc.cell_contour_length((-3.0, 1.0, -3.0, 1.0)) == pytest.approx(math.sqrt(2) / 2)
    # centre mean +1: each segment cuts off an inside corner, legs 1/4
    assert orc.cell_contour_length((-1.0, 3.0, -1.0, 3.0)) == pytest.approx(math.sqrt(2) / 2)
    assert orc.cell_contour_length((3.0, -1.0, 3.0, -1.0)) == pytest.approx(math.sqrt(2) / 2)
    # the other pairing would give legs of 3/4
    assert orc.cell_contour_length((1.0, -3.0, 1.0, -3.0)) == pytest.approx(math.sqrt(2) / 2)
    # one inside corner, crossings at 1/2 on both of its edges
    assert orc.cell_contour_length((-1.0, 1.0, 1.0, 1.0)) == pytest.approx(math.sqrt(0.5))
    # straight cut through the cell; zero counts as outside
    assert orc.cell_contour_length((-1.0, 1.0, 1.0, -1.0)) == pytest.approx(1.0)
    assert orc.cell_contour_length((0.0, 1.0, 1.0, 0.0)) == 0.0
    assert orc.cell_contour_length((-1.0, -1.0, -1.0, -1.0)) == 0.0


def test_contour_is_invariant_under_lattice_symmetries(orc):
    # random field with many saddle cells: transposition, reflections and a
    # periodic shift only relabel the cells (catches corner-order mistakes)
    rng = np.random.default_rng(5)
    phi = rng.uniform(-1, 1, size=(13, 19))
    ref = orc.contour_length(phi, False, False)
    assert orc.contour_length(phi.T.copy(), False, False) == pytest.approx(ref, rel=1e-12)
    assert orc.contour_length(phi[::-1].copy(), False, False) == pytest.approx(ref, rel=1e-12)
    assert orc.contour_length(phi[:, ::-1].copy(), False, False) == pytest.approx(ref, rel=1e-12)
    per = orc.contour_length(phi, True, True)
    shifted = np.roll(np.roll(phi, 5, axis=1), 3, axis=0)
    assert orc.contour_length(shifted, True, True) == pytest.approx(per, rel=1e-12)


@pytest.mark.parametrize("R", [10.3, 20.7, 40.2])
def test_circle_perimeter_converges_to_2_pi_R(orc, R):
    n = int(2 * R + 12)
    x, y = _grid(n, n)
    xc, yc = n / 2 + 0.31, n / 2 - 0.17
    phi = np.hypot(x - xc, y - yc) - R  # signed distance, negative inside
    err = abs(orc.contour_length(phi, False, False) / (2 * math.pi * R) - 1)
    # chords between crossings about one cell apart: relative error O(1/R^2)
    # (measured 0.061 / R^2 at all three radii)
    assert err < 0.08 / R ** 2


def test_ellipse_circularity_against_ramanujan(orc):
    a, b, n = 36.4, 18.3, 100
    x, y = _grid(n, n)
    xc, yc = 50.2, 49.6
    phi = b * (np.hypot((x - xc) / a, (y - yc) / b) - 1.0)
    per = orc.contour_length(phi, False, False)
    h = ((a - b) / (a + b)) ** 2
    ram = math.pi * (a + b) * (1 + 3 * h / (10 + math.sqrt(4 - 3 * h)))
    assert per == pytest.approx(ram, rel=2e-4)
    f = {"phi": phi, "ux": 0 * phi, "uy": 0 * phi}
    out = orc.rising_bubble(f, True, True)
    # lattice-point count of the ellipse: pi a b up to the boundary layer
    assert out["area2"] == pytest.approx(math.pi * a * b, rel=3e-3)
    assert out["circularity"] == pytest.approx(2 * math.sqrt(math.pi * math.pi * a * b) / ram,
                                               rel=3e-3)


def test_centre_of_mass_and_velocity_of_a_sharp_bubble(orc):
    # bubble of phi = -1 at an off-centre node, phi = +1 outside: the weight
    # 1 - phi vanishes outside, so mirror symmetry about the centre fixes the
    # centroid exactly (a 1 + phi weighting would not: the box is lopsided)
    nx, ny, xc, yc, R = 41, 60, 12, 15, 7.5
    x, y = _grid(nx, ny)
    r = np.hypot(x - xc, y - yc)
    phi = np.where(r < R, -1.0, 1.0)
    ux = 0.002 + 0.001 * (x - xc)
    uy = 0.01 + 0.003 * (y - yc) + 0.002 * (x - xc)
    out = orc.rising_bubble({"phi": phi, "ux": ux, "uy": uy}, True, True)
    assert out["xc2"] == pytest.approx(xc, abs=1e-12)
    assert out["yc2"] == pytest.approx(yc, abs=1e-12)
    assert out["uc2"] == pytest.approx(0.002, abs=1e-15)
    assert out["vc2"] == pytest.approx(0.01, abs=1e-15)
    # brute-force lattice-point count of the open disk
    count = sum(1 for i in range(-8, 9) for j in range(-8, 9) if i * i + j * j < R * R)
    assert out["area2"] == count and out["mass2"] == pytest.approx(2 * count)


def test_tanh_bubble_quantities(orc):
    from paper_2012_14729_gb300 import workloads as wl
    nx, ny, R = 120, 240, 30.0
    phi = wl.bubble(nx, ny, R, 4.0, xc=59.5, yc=59.5)
    f = {"phi": phi, "ux": 0 * phi, "uy": 0 * phi}
    out = orc.rising_bubble(f, True, True)
    assert out["yc2"] == pytest.approx(59.5, abs=1e-9)
    assert out["xc2"] == pytest.approx(59.5, abs=1e-9)
    assert out["perimeter"] == pytest.approx(2 * math.pi * R, rel=1e-4)
    assert out["circularity"] == pytest.approx(1.0, abs=2e-3)


def test_no_interface(orc):
    phi = np.ones((8, 9))
    out = orc.rising_bubble({"phi": phi, "ux": 0 * phi, "uy": 0 * phi}, False, False)
    assert out["perimeter"] == 0.0 and out["circularity"] == 0.0 and out["area2"] == 0.0

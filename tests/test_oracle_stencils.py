"""Oracle pins: the isotropic central scheme (Eqs. ICS-1st, ICS-sec) and the
wall ghost rule.

Pinned by facts independent of the stencil's code: exact derivatives of low
degree polynomials, second-order convergence on smooth periodic fields, the
telescoping of a central difference over a periodic grid, and the definition
of the wall ghosts as an even reflection about the wall plane (built here by
explicitly mirroring the field into a periodic grid twice as tall).
"""
import math

import numpy as np
import pytest


def _poly_grid(n, fn):
    y, x = np.mgrid[0:n, 0:n].astype(float)
    x -= n / 2
    y -= n / 2
    return x, y, fn(x, y)


@pytest.mark.parametrize("deg", [1, 2, 3])
def test_gradient_exact_on_cubics(orc, deg):
    rng = np.random.default_rng(deg)
    c = rng.uniform(-1, 1, 10)
    def f(x, y):
        v = c[0] + c[1] * x + c[2] * y
        if deg >= 2:
            v = v + c[3] * x * x + c[4] * x * y + c[5] * y * y
        if deg >= 3:
            v = v + c[6] * x ** 3 + c[7] * x * x * y + c[8] * x * y * y + c[9] * y ** 3
        return v * 1e-3
    n = 16
    x, y, a = _poly_grid(n, f)
    gx, gy, _ = orc.ics(a)
    ex_gx = c[1] + 2 * c[3] * x + c[4] * y
    ex_gy = c[2] + c[4] * x + 2 * c[5] * y
    if deg < 2:
        ex_gx = np.full_like(x, c[1])
        ex_gy = np.full_like(x, c[2])
    if deg >= 3:
        ex_gx = ex_gx + 3 * c[6] * x * x + 2 * c[7] * x * y + c[8] * y * y
        ex_gy = ex_gy + c[7] * x * x + 2 * c[8] * x * y + 3 * c[9] * y * y
    ex_gx *= 1e-3
    ex_gy *= 1e-3
    sl = (slice(1, n - 1), slice(1, n - 1))  # away from the periodic seam
    # cubic terms: the central sum over the D2Q9 links adds the lattice's
    # fourth moments, sum w c_x^4 = 1/3 and sum w c_x^2 c_y^2 = 1/9, so
    # grad_x(x^3) = 3x^2 + 1 and grad_x(x y^2) = y^2 + 1/3 (likewise in y)
    if deg >= 3:
        ex_gx = ex_gx + 1e-3 * (c[6] * 1.0 + c[8] * (1.0 / 3.0))
        ex_gy = ex_gy + 1e-3 * (c[9] * 1.0 + c[7] * (1.0 / 3.0))
    np.testing.assert_allclose(gx[sl], ex_gx[sl], atol=1e-14)
    np.testing.assert_allclose(gy[sl], ex_gy[sl], atol=1e-14)


def test_laplacian_exact_on_quadratics(orc):
    rng = np.random.default_rng(7)
    c = rng.uniform(-1, 1, 6)
    n = 16
    x, y, a = _poly_grid(n, lambda x, y: c[0] + c[1] * x + c[2] * y + c[3] * x * x
                         + c[4] * x * y + c[5] * y * y)
    _, _, lap = orc.ics(a)
    sl = (slice(1, n - 1), slice(1, n - 1))
    np.testing.assert_allclose(lap[sl], 2 * c[3] + 2 * c[5], atol=1e-12)


def test_second_order_convergence(orc):
    """On a smooth periodic field the stencils converge to the exact
    derivatives at second order."""
    errs = []
    for n in (32, 64, 128):
        h = 1.0 / n
        y, x = np.mgrid[0:n, 0:n].astype(float) * h
        k = 2 * math.pi
        a = np.sin(k * x) * np.cos(2 * k * y)
        gx, gy, lap = orc.ics(a)
        # lattice derivatives are per cell: rescale by 1/h
        e_gx = np.abs(gx / h - k * np.cos(k * x) * np.cos(2 * k * y)).max()
        e_gy = np.abs(gy / h + 2 * k * np.sin(k * x) * np.sin(2 * k * y)).max()
        e_l = np.abs(lap / h ** 2 + 5 * k * k * a).max()
        errs.append((e_gx, e_gy, e_l))
    for a, b in zip(errs[:-1], errs[1:]):
        for ea, eb in zip(a, b):
            assert 3.6 < ea / eb < 4.4


def test_gradient_telescopes_on_periodic_grid(orc):
    rng = np.random.default_rng(3)
    a = rng.standard_normal((12, 20))
    gx, gy, lap = orc.ics(a)
    assert abs(gx.sum()) < 1e-12 and abs(gy.sum()) < 1e-12 and abs(lap.sum()) < 1e-12


def test_isotropy_of_laplacian(orc):
    """Plane waves of equal |k| along an axis and along a diagonal see the
    same Laplacian up to O(k^4) (the scheme is isotropic to second order)."""
    n = 256
    y, x = np.mgrid[0:n, 0:n].astype(float)
    k = 2 * math.pi * 8 / n
    a1 = np.cos(k * math.sqrt(2) * x)          # |k| = sqrt(2) k along x
    a2 = np.cos(k * (x + y))                   # same |k| along the diagonal
    l1 = orc.ics(a1)[2][5, 5] / a1[5, 5]
    l2 = orc.ics(a2)[2][5, 5] / a2[5, 5]
    kk = 2 * k * k
    assert abs(l1 + kk) / kk < 0.05 and abs(l2 + kk) / kk < 0.05
    assert abs(l1 - l2) / kk < (kk ** 2) * 0.05


@pytest.mark.parametrize("ny", [5, 8, 13])
def test_wall_ghosts_are_even_reflection(orc, ny):
    """With walls at y = -1/2 and y = ny - 1/2 the stencils see the field
    reflected about each wall plane.  Mirror the field explicitly into a
    periodic grid of 2 ny rows: the periodic stencils there must equal the
    walled stencils on the original rows."""
    rng = np.random.default_rng(ny)
    a = rng.standard_normal((ny, 7))
    ext = np.concatenate([a, a[::-1]], axis=0)   # rows ny..2ny-1 mirror the top wall
    gx_w, gy_w, l_w = orc.ics(a, wall=True)
    gx_p, gy_p, l_p = orc.ics(ext)
    np.testing.assert_allclose(gx_w, gx_p[:ny], atol=1e-14)
    np.testing.assert_allclose(gy_w, gy_p[:ny], atol=1e-14)
    np.testing.assert_allclose(l_w, l_p[:ny], atol=1e-14)

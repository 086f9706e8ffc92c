"""Oracle pins for free-slip (mirror-symmetry) side walls at x = -1/2 and
x = nx - 1/2, the boundary of the rising-bubble benchmark (Sec. 5.4):

  - an x-independent state with an x-independent force never feels the
    side walls: it evolves exactly as on the periodic-x grid, which is pinned
    on its own (a specular reflection at the walls produces no shear);
  - sum phi is conserved exactly, with and without no-slip walls in y;
  - a drop against the left wall, centred on it, is half of a drop centred
    at x = 0 on the periodic grid of twice the width (the symmetry plane);
  - the symmetry plane admits no x-forcing: gravity along x and moving
    no-slip walls in y (both odd under the mirror) are refused.
"""
import numpy as np
import pytest

from paper_2012_14729_gb300 import workloads as wl

FORMS = ("STF1", "STF2", "CPF1", "CPF2", "PF1", "PF2", "CSF1", "CSF2")


def _par(orc, form, **kw):
    base = dict(sigma=0.01, W=4.0, M=0.1, rho1=1.0, rho2=0.5, nu1=0.1, nu2=0.05, form=form)
    return orc.Params(**{**base, **kw})


@pytest.mark.parametrize("wall_y", [False, True])
@pytest.mark.parametrize("form", ["STF1", "CPF1", "CSF2"])
def test_x_independent_state_ignores_the_side_walls(orc, form, wall_y):
    nx, ny = 12, 40
    y = np.arange(ny)[:, None] + np.zeros((1, nx))
    phi0 = np.tanh(2 * (20.3 - y) / 4.0)          # a flat interface across x
    par = _par(orc, form, gy=-2e-5)
    a = orc.Sim(nx, ny, wall_y, par, phi0, wall_x=True).step(60)
    b = orc.Sim(nx, ny, wall_y, par, phi0, wall_x=False).step(60)
    np.testing.assert_allclose(a.f, b.f, atol=1e-13, rtol=0)
    np.testing.assert_allclose(a.h, b.h, atol=1e-13, rtol=0)


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("wall_y", [False, True])
def test_mass_conserved_with_side_walls(orc, form, wall_y):
    nx, ny = 30, 26
    phi0 = wl.drop(nx, ny, 7.0, 4.0, xc=4.3, yc=11.2, periodic_y=not wall_y)
    par = _par(orc, form, gy=-1e-5)
    s = orc.Sim(nx, ny, wall_y, par, phi0, wall_x=True)
    m0 = s.macro()["phi"].sum()
    s.step(200)
    m1 = s.macro()["phi"].sum()
    assert abs(m1 - m0) <= 1e-11 * np.abs(s.macro()["phi"]).sum()


@pytest.mark.parametrize("form", ["STF2", "PF2", "CSF1"])
def test_drop_on_the_wall_is_half_a_drop(orc, form):
    """Drop centred on the wall plane x = -1/2 of an nx-wide grid with side
    walls = the left half (x < nx) of a drop centred at x = -1/2 (i.e. at
    2 nx - 1/2) on the periodic grid of width 2 nx."""
    nx, ny = 20, 28
    par = _par(orc, form)
    phi_w = wl.drop(2 * nx, ny, 8.0, 4.0, xc=-0.5, yc=13.7)       # periodic distance
    a = orc.Sim(nx, ny, False, par, phi_w[:, :nx], wall_x=True).step(40)
    b = orc.Sim(2 * nx, ny, False, par, phi_w, wall_x=False).step(40)
    fa, fb = a.macro(), b.macro()
    for k in ("phi", "ux", "uy", "P"):
        np.testing.assert_allclose(fa[k], fb[k][:, :nx], atol=1e-12, rtol=0, err_msg=k)


def test_x_forcing_is_refused(orc):
    phi0 = np.ones((8, 8))
    for kw in (dict(gx=1e-5), dict(uw_bottom=0.01)):
        with pytest.raises(ValueError):
            orc.Sim(8, 8, True, _par(orc, "STF1", **kw), phi0, wall_x=True)

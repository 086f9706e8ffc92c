"""GPU parity of pflbm_bubble_diagnostics, the rising-bubble quantities of
Sec. 5.4 (Eqs. quantify-yc, quantify-uc, circularity), against the oracle.

Two comparisons: (1) on the same float32 fields (the GPU's own read-back,
widened to FP64), where both sides take every inside/outside and saddle
decision on the same values, so the node count is equal and the sums agree to
FP64 summation order; (2) on the oracle's own state after the same steps,
within what the state tolerance moves the contour."""
import math

import numpy as np
import pytest

from paper_2012_14729_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

SUMS = ("mass2", "xc2", "yc2", "uc2", "vc2", "perimeter", "circularity")


@pytest.fixture(scope="module")
def pf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2012_14729_gb300 import build, pflbm
    build.build()
    pflbm.load()
    return pflbm


def _same_fields(pf, orc, d, wall_x, wall_y):
    g = d.bubble_diagnostics()
    f = {k: v.astype(np.float64) for k, v in d.fields().items()}
    o = orc.rising_bubble(f, wall_x, wall_y)
    assert g["area2"] == o["area2"]
    for k in SUMS:
        assert abs(g[k] - o[k]) <= 1e-11 * max(1.0, abs(o[k])), (k, g[k], o[k])
    return g, o


def _domain(pf, nx, ny, wall_y, wall_x, p, phi0):
    d = pf.Domain(nx, ny, wall_y=wall_y, wall_x=wall_x).set_params(**p)
    d.init_phi(phi0.astype(np.float32))
    return d


def test_rising_bubble_same_fields_and_oracle_state(pf, orc):
    c = wl.rising_bubble("STF1", nx=120)
    d = _domain(pf, c.nx, c.ny, True, True, c.params, c.phi0)
    d.step(400)
    g, _ = _same_fields(pf, orc, d, True, True)
    assert g["status"] == "PFLBM_OK" and g["vc2"] > 0 and g["perimeter"] > 150
    s = orc.Sim(c.nx, c.ny, True, orc.Params(**c.params),
                c.phi0.astype(np.float32).astype(np.float64), wall_x=True).step(400)
    m = s.macro()
    o = orc.rising_bubble(m, True, True)
    f = d.fields()
    e_phi = float(np.abs(f["phi"] - m["phi"]).max())
    e_u = float(np.abs(f["uy"] - m["uy"]).max())
    # state bar: 1e-5 / 1e-6, or 5x the deviation of the oracle's algorithm
    # with float32 state where that is larger (density ratio 10 at the walls)
    dev = orc.float32_deviation(c.nx, c.ny, True, orc.Params(**c.params),
                                c.phi0.astype(np.float32).astype(np.float64), 400, wall_x=True)
    assert e_phi <= max(1e-5, 5 * dev["phi"]) and e_u <= max(1e-6, 5 * dev["u"]), (e_phi, e_u)
    # phi within e_phi moves a crossing by ~e_phi / |grad phi| (~2e-5 cells)
    assert abs(g["area2"] - o["area2"]) <= 1
    assert g["perimeter"] == pytest.approx(o["perimeter"], rel=1e-4)
    # the weighted means move by at most what the node errors allow:
    # y_c = sum w y / sum w with w = 1 - phi off by <= e_phi at every node
    y = np.arange(c.ny, dtype=np.float64)[:, None] + 0 * m["phi"]
    den = o["mass2"] - e_phi * y.size
    tol_y = e_phi * np.abs(y - o["yc2"]).sum() / den
    tol_v = (e_phi * np.abs(m["uy"] - o["vc2"]).sum() + e_u * o["mass2"]) / den
    assert abs(g["yc2"] - o["yc2"]) <= 1.01 * tol_y, (g["yc2"], o["yc2"], tol_y)
    assert abs(g["vc2"] - o["vc2"]) <= 1.01 * tol_v, (g["vc2"], o["vc2"], tol_v)


@pytest.mark.parametrize("nx,ny,wall_y", [(97, 61, False), (97, 61, True), (4, 4, False),
                                          (300, 7, True)])
def test_saddles_and_wrapped_cells(pf, orc, nx, ny, wall_y):
    # a smooth random field of both signs: many contours, saddle cells,
    # contours crossing the periodic edges; ragged block tails
    phi0 = wl.smooth_random(nx, ny, seed=nx + ny, modes=4, amp=0.9)
    phi0 = np.clip(phi0 + wl.noise(nx, ny, 0.05, seed=3), -1, 1)
    p = dict(sigma=0.01, W=4.0, M=0.1, rho1=1.0, rho2=1.0, nu1=0.1, nu2=0.1, form="STF1")
    d = _domain(pf, nx, ny, wall_y, False, p, phi0)
    g, _ = _same_fields(pf, orc, d, False, wall_y)
    d.step(3)
    _same_fields(pf, orc, d, False, wall_y)
    assert g["perimeter"] > 0


def test_drop_across_the_periodic_corner(pf, orc):
    # bubble centred on the corner of a doubly periodic box: every contour
    # cell in the wrap rows and columns takes part
    nx, ny = 64, 48
    dx, dy = wl._dist(nx, ny, 0.3, 0.6)
    phi0 = -np.tanh(2.0 * (12.0 - np.hypot(dx, dy)) / 4.0)
    p = dict(sigma=0.01, W=4.0, M=0.1, rho1=1.0, rho2=1.0, nu1=0.1, nu2=0.1, form="STF1")
    d = _domain(pf, nx, ny, False, False, p, phi0)
    g, _ = _same_fields(pf, orc, d, False, False)
    assert g["perimeter"] == pytest.approx(2 * math.pi * 12.0, rel=2e-3)
    assert g["circularity"] == pytest.approx(1.0, abs=5e-3)


def test_side_walls_cut_the_cells(pf, orc):
    # free-slip side walls: no cell joins column nx-1 to column 0, so a
    # bubble against the left wall is open there
    nx, ny = 70, 45
    dx, dy = wl._dist(nx, ny, 3.0, 20.0, False, False)
    phi0 = -np.tanh(2.0 * (10.0 - np.hypot(dx, dy)) / 4.0)
    p = dict(sigma=0.01, W=4.0, M=0.1, rho1=1.0, rho2=0.5, nu1=0.1, nu2=0.1, gy=-1e-5,
             form="CSF1")
    d = _domain(pf, nx, ny, True, True, p, phi0)
    d.step(50)
    g, _ = _same_fields(pf, orc, d, True, True)
    assert g["perimeter"] < 2 * math.pi * 10.0


def test_no_interface_and_nonfinite(pf):
    nx, ny = 40, 30
    p = dict(sigma=0.01, W=4.0, M=0.1, rho1=1.0, rho2=1.0, nu1=0.1, nu2=0.1, form="STF1")
    d = _domain(pf, nx, ny, True, False, p, np.ones((ny, nx)))
    g = d.bubble_diagnostics()
    assert g["status"] == "PFLBM_OK"
    assert g["perimeter"] == 0 and g["circularity"] == 0 and g["area2"] == 0
    assert g["mass2"] == pytest.approx(0.0, abs=1e-3)
    bad = wl.bubble(nx, ny, 8.0, 4.0)
    bad[5, 7] = np.nan
    d = _domain(pf, nx, ny, True, False, p, bad)
    g = d.bubble_diagnostics()
    assert g["status"] == "PFLBM_EUNSTABLE" and g["nonfinite"] >= 1

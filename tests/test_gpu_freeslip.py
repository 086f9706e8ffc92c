"""GPU parity with free-slip side walls (x = -1/2 and nx - 1/2, the
rising-bubble boundary of Sec. 5.4) against the FP64 oracle, whose side walls
are the mirror-doubled periodic domain written out: every force form, with
periodic or no-slip (resting) walls in y, a drop touching a side wall, grids
that leave partial tiles, and the same bar as the other parity tests."""
import numpy as np
import pytest

from paper_2012_14729_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FORMS = ("STF1", "STF2", "CPF1", "CPF2", "PF1", "PF2", "CSF1", "CSF2")
TOL_PHI, TOL_U = 1e-5, 1e-6


@pytest.fixture(scope="module")
def pf():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2012_14729_gb300 import build, pflbm
    build.build()
    pflbm.load()
    return pflbm


def _pair(pf, orc, nx, ny, wall_y, p, phi0, steps):
    d = pf.Domain(nx, ny, wall_y=wall_y, wall_x=True).set_params(**p)
    d.init_phi(phi0.astype(np.float32))
    d.step(steps)
    g = d.fields()
    s = orc.Sim(nx, ny, wall_y, orc.Params(**p), phi0.astype(np.float32).astype(np.float64),
                wall_x=True).step(steps)
    return g, s.macro(), d


def _err(g, o, k):
    return float(np.abs(g[k].astype(np.float64) - o[k]).max())


@pytest.mark.parametrize("wall_y", [False, True])
@pytest.mark.parametrize("form", FORMS)
def test_side_walls_match_the_oracle(pf, orc, form, wall_y):
    """70 x 45: partial tiles in x and y; the drop's interface crosses the
    left wall; gravity along y and a density contrast."""
    nx, ny = 70, 45
    phi0 = wl.drop(nx, ny, 10.0, 4.0, xc=4.3, yc=21.6, periodic_y=not wall_y)
    p = dict(sigma=0.01, W=4.0, M=0.1, rho1=1.0, rho2=0.25, nu1=0.1, nu2=0.2, gy=-1e-5,
             form=form)
    g, o, _ = _pair(pf, orc, nx, ny, wall_y, p, phi0, 300)
    e = (_err(g, o, "phi"), _err(g, o, "ux"), _err(g, o, "uy"))
    assert e[0] <= TOL_PHI and max(e[1:]) <= TOL_U, e


def test_wide_grid_with_inner_tiles(pf, orc):
    """200 x 120 with y walls: inner tiles between the side-wall tiles, two
    drops, one against each side wall.  Tolerance: the fixed bar or 5x the
    deviation of the oracle's own algorithm run with float32 state
    (oracle.float32_deviation), which on this wall-and-gravity case moves
    phi by more than 1e-5 by itself."""
    nx, ny = 200, 120
    phi0 = np.maximum(wl.drop(nx, ny, 14.0, 4.0, xc=8.0, yc=50.0, periodic_y=False),
                      wl.drop(nx, ny, 12.0, 4.0, xc=193.0, yc=70.0, periodic_y=False))
    p = dict(sigma=0.01, W=4.0, M=0.1, rho1=1.0, rho2=0.5, nu1=0.1, nu2=0.1, gy=-2e-5,
             form="STF1")
    g, o, d = _pair(pf, orc, nx, ny, True, p, phi0, 200)
    dev = orc.float32_deviation(nx, ny, True, orc.Params(**p),
                                phi0.astype(np.float32).astype(np.float64), 200, wall_x=True)
    tol_phi, tol_u = max(TOL_PHI, 5 * dev["phi"]), max(TOL_U, 5 * dev["u"])
    e = (_err(g, o, "phi"), _err(g, o, "ux"), _err(g, o, "uy"))
    assert e[0] <= tol_phi and max(e[1:]) <= tol_u, (e, dev["phi"], dev["u"])
    # the populations themselves, through the specular pulls of the read-back
    fo = orc.Sim(nx, ny, True, orc.Params(**p), phi0.astype(np.float32).astype(np.float64),
                 wall_x=True).step(200)
    f, h = d.populations()
    assert float(np.abs(h - fo.h).max()) <= tol_phi
    assert float(np.abs(f - fo.f).max()) <= 2 * tol_u


def test_side_walls_refuse_x_forcing_and_boxes(pf):
    d = pf.Domain(40, 40, wall_y=True, wall_x=True)
    with pytest.raises(pf.PflbmError):
        d.set_params(sigma=0.01, gx=1e-5)
    with pytest.raises(pf.PflbmError):
        d.set_params(sigma=0.01, uw_top=0.01)
    d.set_params(sigma=0.01)
    with pytest.raises(pf.PflbmError):
        d.stage_mode("boxes")
    d.init_phi(wl.drop(40, 40, 8.0, 4.0, periodic_y=False).astype(np.float32))
    # side walls are staged by gathers (32 x 16 or 32 x 8 tiles) only
    assert d.autotune(2) in ("gather", "gather8")


@pytest.mark.parametrize("storage,tol_phi,tol_u", [("fp16", 2e-4, 2e-5), ("bf16", 2e-3, 2e-4)])
def test_side_walls_with_16bit_storage(pf, orc, storage, tol_phi, tol_u):
    """16-bit population storage through the specular pulls: error against
    the FP64 oracle at the 16-bit bars of the periodic storage tests."""
    nx, ny = 70, 45
    phi0 = wl.drop(nx, ny, 10.0, 4.0, xc=4.3, yc=21.6, periodic_y=False)
    p = dict(sigma=0.01, W=4.0, M=0.1, rho1=1.0, rho2=0.25, nu1=0.1, nu2=0.2, gy=-1e-5,
             form="CSF1")
    d = pf.Domain(nx, ny, wall_y=True, wall_x=True, storage=storage).set_params(**p)
    d.init_phi(phi0.astype(np.float32))
    d.step(200)
    g = d.fields()
    o = orc.Sim(nx, ny, True, orc.Params(**p), phi0.astype(np.float32).astype(np.float64),
                wall_x=True).step(200).macro()
    e = (_err(g, o, "phi"), _err(g, o, "ux"), _err(g, o, "uy"))
    assert e[0] <= tol_phi and max(e[1:]) <= tol_u, e


def test_side_walls_state_round_trip_and_refusals(pf):
    nx, ny = 48, 40
    p = dict(sigma=0.01, W=4.0, M=0.1, rho1=1.0, rho2=0.5, nu1=0.1, nu2=0.1, gy=-1e-5)
    phi0 = wl.drop(nx, ny, 8.0, 4.0, xc=3.0, yc=20.0, periodic_y=False).astype(np.float32)
    a = pf.Domain(nx, ny, wall_y=True, wall_x=True).set_params(**p).init_phi(phi0)
    a.step(20)
    blob = a.save_state()
    a.step(30)
    b = pf.Domain(nx, ny, wall_y=True, wall_x=True).set_params(**p).load_state(blob)
    b.step(30)
    for k, v in a.fields().items():
        np.testing.assert_array_equal(v, b.fields()[k])
    # a side-wall state does not load into a periodic-x domain
    c = pf.Domain(nx, ny, wall_y=True).set_params(**p)
    with pytest.raises(pf.PflbmError):
        c.load_state(blob)
    # the batch and the adjoint take periodic x only
    with pytest.raises(pf.PflbmError):
        pf.Batch([a])
    assert pf.pflbm_adjoint_scratch_bytes(a.h, 10, 5) == 0


@pytest.mark.parametrize("form", ["STF1", "CSF2"])
def test_x_independent_state_ignores_the_side_walls(pf, form):
    """A flat interface (phi independent of x) under gravity along y never
    feels mirror planes in x: the side-wall run equals the periodic run to
    float32 rounding (separately compiled kernels)."""
    nx, ny = 70, 45
    y = np.arange(ny, dtype=np.float64)[:, None] + np.zeros((1, nx))
    phi0 = np.tanh(2.0 * (20.3 - y) / 4.0).astype(np.float32)
    p = dict(sigma=0.01, W=4.0, M=0.1, rho1=1.0, rho2=0.25, nu1=0.1, nu2=0.2, gy=-1e-5,
             form=form)
    out = []
    for wall_x in (True, False):
        d = pf.Domain(nx, ny, wall_y=True, wall_x=wall_x).set_params(**p).init_phi(phi0)
        d.step(300)
        out.append(d.fields())
    for k in ("phi", "ux", "uy", "P"):
        scale = float(np.abs(out[1][k]).max()) + 1e-12
        assert float(np.abs(out[0][k] - out[1][k]).max()) <= 1e-5 * scale, k
    assert float(np.abs(out[0]["ux"]).max()) <= 1e-6


def test_side_walls_graph_replay_equals_plain_launches(pf):
    nx, ny = 70, 45
    phi0 = wl.drop(nx, ny, 10.0, 4.0, xc=4.3, yc=21.6, periodic_y=False).astype(np.float32)
    p = dict(sigma=0.01, W=4.0, M=0.1, rho1=1.0, rho2=0.25, nu1=0.1, nu2=0.2, gy=-1e-5)
    out = []
    for graphs in (False, True):
        d = pf.Domain(nx, ny, wall_y=True, wall_x=True).set_params(**p).init_phi(phi0)
        d.graphs(graphs)
        d.step(3)
        d.step(40)
        out.append(d.populations())
    for a, b in zip(out[0], out[1]):
        np.testing.assert_array_equal(a, b)

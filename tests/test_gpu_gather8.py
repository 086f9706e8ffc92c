"""GPU tests of the short-tile gather mode (PFLBM_STAGE_GATHER8: 256-thread
CTAs per 32 x 8 tile, one collision node per thread, each thread pulling its
own node first in passes 1 and 3 and colliding it from registers): parity
with the FP64 oracle
at the plain-step bar for every force form on periodic, walled-and-ragged and
side-walled lattices; equality with the two-node gather mode for every
storage format (the per-node arithmetic is the same, only the order in which
a CTA visits its nodes differs); the 16-bit bars against the oracle; graph
replay and the autotuner's choice among all modes."""
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


def _gpu(pf, nx, ny, p, phi0, steps, stage, wall=False, wall_x=False, storage="fp32",
         graphs=False):
    d = pf.Domain(nx, ny, wall_y=wall, wall_x=wall_x, storage=storage).set_params(**p)
    d.stage_mode(stage)
    if graphs:
        d.graphs(True)
    d.init_phi(phi0.astype(np.float32))
    d.step(steps)
    assert d.diagnostics()["status"] == "PFLBM_OK"
    return d


def _oracle(orc, nx, ny, p, phi0, steps, wall=False, wall_x=False):
    s = orc.Sim(nx, ny, wall, orc.Params(**p), phi0.astype(np.float32).astype(np.float64),
                wall_x=wall_x)
    return s.step(steps).macro()


def _errs(g, o):
    e_phi = float(np.abs(g["phi"] - o["phi"]).max())
    e_u = float(max(np.abs(g["ux"] - o["ux"]).max(), np.abs(g["uy"] - o["uy"]).max()))
    return e_phi, e_u


@pytest.mark.parametrize("form", FORMS)
def test_gather8_stationary_drop_1000_steps(pf, orc, form):
    c = wl.stationary_drop(form)
    d = _gpu(pf, c.nx, c.ny, c.params, c.phi0, 1000, "gather8")
    assert d.stage() == "gather8"
    e_phi, e_u = _errs(d.fields(), _oracle(orc, c.nx, c.ny, c.params, c.phi0, 1000))
    assert e_phi <= TOL_PHI and e_u <= TOL_U, (e_phi, e_u)


@pytest.mark.parametrize("form", FORMS)
def test_gather8_walls_ragged(pf, orc, form):
    """100 x 37: partial tiles in x (100 = 3 x 32 + 4) and y (37 = 4 x 8 +
    5), walls moving at -/+0.01, gravity, density ratio 4, viscosity ratio
    2, a drop near the bottom wall."""
    nx, ny = 100, 37
    phi0 = wl.drop(nx, ny, 9.0, 4.0, xc=61.3, yc=11.2, periodic_y=False)
    p = dict(sigma=0.01, W=4.0, M=0.1, rho1=1.0, rho2=0.25, nu1=0.1, nu2=0.2,
             gy=-1e-5, uw_bottom=-0.01, uw_top=0.01, form=form)
    d = _gpu(pf, nx, ny, p, phi0, 300, "gather8", wall=True)
    e_phi, e_u = _errs(d.fields(), _oracle(orc, nx, ny, p, phi0, 300, wall=True))
    assert e_phi <= TOL_PHI and e_u <= TOL_U, (e_phi, e_u)


@pytest.mark.parametrize("wall_y", [False, True])
@pytest.mark.parametrize("form", ["STF1", "CPF2", "PF2", "CSF1"])
def test_gather8_side_walls(pf, orc, form, wall_y):
    """70 x 45 with free-slip side walls: partial tiles, the drop's interface
    crosses the left wall."""
    nx, ny = 70, 45
    phi0 = wl.drop(nx, ny, 10.0, 4.0, xc=4.3, yc=21.6, periodic_y=not wall_y)
    p = dict(sigma=0.01, W=4.0, M=0.1, rho1=1.0, rho2=0.25, nu1=0.1, nu2=0.2, gy=-1e-5,
             form=form)
    d = _gpu(pf, nx, ny, p, phi0, 300, "gather8", wall=wall_y, wall_x=True)
    e_phi, e_u = _errs(d.fields(), _oracle(orc, nx, ny, p, phi0, 300, wall=wall_y, wall_x=True))
    assert e_phi <= TOL_PHI and e_u <= TOL_U, (e_phi, e_u)


def _case(wall):
    nx, ny = 256, 128
    phi0 = wl.two_drops(nx, ny, 25.0, 25.0, 2.0, 5.0) if not wall else \
        wl.drop(nx, ny, 30.0, 5.0, xc=100.3, yc=60.7, periodic_y=False)
    p = dict(sigma=1e-3, W=5.0, M=0.05, rho1=1.0, rho2=0.2, nu1=0.1, nu2=0.1,
             gy=-1e-6 if wall else 0.0, uw_bottom=-0.005 if wall else 0.0,
             uw_top=0.005 if wall else 0.0)
    return nx, ny, phi0, p


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("wall", [False, True])
@pytest.mark.parametrize("form", ["STF1", "CPF1", "PF2", "CSF2"])
def test_gather8_equals_gather(pf, storage, wall, form):
    """Same populations as the two-node gather mode after 60 steps.  Each
    node runs the same expressions in both kernels, so the populations agree
    to the compiler's multiply-add contraction of two separately compiled
    kernels (16-bit: one unit in the last place where a value lands on the
    other side of a rounding boundary); the largest difference is printed."""
    nx, ny, phi0, p = _case(wall)
    p["form"] = form
    out = [_gpu(pf, nx, ny, p, phi0, 60, st, wall=wall, storage=storage).populations()
           for st in ("gather", "gather8")]
    worst = 0.0
    for a, b in zip(out[0], out[1]):
        scale = float(np.abs(a).max())
        worst = max(worst, float(np.abs(a.astype(np.float64) - b).max()) / scale)
    print(f"GATHER8=GATHER {form} {storage} walls={wall}: largest difference / scale {worst:.2e}")
    assert worst <= {"fp32": 2e-5, "fp16": 2e-3, "bf16": 1e-2}[storage], worst


@pytest.mark.parametrize("wall", [False, True])
@pytest.mark.parametrize("storage,tol_phi,tol_u", [("fp16", 2e-4, 2e-5), ("bf16", 2e-3, 2e-4)])
def test_gather8_16bit_against_oracle(pf, orc, storage, tol_phi, tol_u, wall):
    nx, ny, phi0, p = _case(wall)
    p["form"] = "STF1"
    d = _gpu(pf, nx, ny, p, phi0, 200, "gather8", wall=wall, storage=storage)
    e_phi, e_u = _errs(d.fields(), _oracle(orc, nx, ny, p, phi0, 200, wall=wall))
    assert e_phi <= tol_phi and e_u <= tol_u, (e_phi, e_u)


def test_gather8_graphs_equal_plain_launches(pf):
    nx, ny, phi0, p = _case(True)
    a = _gpu(pf, nx, ny, p, phi0, 40, "gather8", wall=True).populations()
    b = _gpu(pf, nx, ny, p, phi0, 40, "gather8", wall=True, graphs=True).populations()
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_autotune_considers_gather8_and_keeps_state(pf):
    nx, ny, phi0, p = _case(False)
    d = pf.Domain(nx, ny, wall_y=False).set_params(**p).init_phi(phi0.astype(np.float32))
    d.step(5)
    before = d.populations()
    mode = d.autotune(3)
    assert mode in ("boxes", "gather", "march", "gather8")
    after = d.populations()
    for x, y in zip(before, after):
        assert np.array_equal(x, y)
    # side walls: only the gather modes
    s = pf.Domain(70, 45, wall_y=True, wall_x=True).set_params(sigma=0.01, W=4.0, M=0.1)
    s.init_phi(wl.drop(70, 45, 10.0, 4.0, xc=4.3, yc=21.6, periodic_y=False).astype(np.float32))
    assert s.autotune(2) in ("gather", "gather8")

"""GPU tests of the marching stage mode (persistent CTAs sweep column strips
along y, staging the pulled population rows ahead into a shared-memory ring
of row slots): parity with the FP64 oracle at the plain-step bar, equality
with the gather mode to float32 rounding for every storage format, the
16-bit bars, lattices whose CTA shares split at strip boundaries, graph
replay, and the cases the mode refuses."""
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


def _gpu(pf, nx, ny, wall, p, phi0, steps, stage, storage="fp32", graphs=False):
    d = pf.Domain(nx, ny, wall_y=wall, storage=storage).set_params(**p)
    d.stage_mode(stage)
    if graphs:
        d.graphs(True)
    d.init_phi(phi0.astype(np.float32))
    d.step(steps)
    assert d.diagnostics()["status"] == "PFLBM_OK"
    return d


def _oracle(orc, nx, ny, wall, p, phi0, steps):
    s = orc.Sim(nx, ny, wall, orc.Params(**p), phi0.astype(np.float32).astype(np.float64))
    return s.step(steps).macro()


def _errs(g, o):
    e_phi = float(np.abs(g["phi"] - o["phi"]).max())
    e_u = float(max(np.abs(g["ux"] - o["ux"]).max(), np.abs(g["uy"] - o["uy"]).max()))
    return e_phi, e_u


@pytest.mark.parametrize("form", FORMS)
def test_march_stationary_drop_1000_steps(pf, orc, form, march="march"):
    c = wl.stationary_drop(form)
    d = _gpu(pf, c.nx, c.ny, False, c.params, c.phi0, 1000, march)
    assert d.stage() == march
    e_phi, e_u = _errs(d.fields(), _oracle(orc, c.nx, c.ny, False, c.params, c.phi0, 1000))
    assert e_phi <= TOL_PHI and e_u <= TOL_U, (e_phi, e_u)


@pytest.mark.parametrize("form", FORMS)
def test_march_walls_ragged(pf, orc, form, march="march"):
    """100 x 37: a strip of 36 columns after one of 64, rows not a multiple
    of the 4 per iteration; walls moving at -/+0.01, gravity, density ratio
    4, viscosity ratio 2, a drop near the bottom wall."""
    nx, ny = 100, 37
    phi0 = wl.drop(nx, ny, 9.0, 4.0, xc=61.3, yc=11.2, periodic_y=False)
    p = dict(sigma=0.01, W=4.0, M=0.1, rho1=1.0, rho2=0.25, nu1=0.1, nu2=0.2,
             gy=-1e-5, uw_bottom=-0.01, uw_top=0.01, form=form)
    d = _gpu(pf, nx, ny, True, p, phi0, 300, march)
    e_phi, e_u = _errs(d.fields(), _oracle(orc, nx, ny, True, p, phi0, 300))
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
def test_march_equals_gather(pf, storage, wall, form, march="march"):
    """Same populations as the gather mode after 60 steps, to float32
    rounding (the two kernels are compiled separately and may contract
    multiply-adds differently; a 16-bit value that lands on the other side of
    a rounding boundary differs by one unit in the last place, 2^-11 of its
    scale for FP16 and 2^-8 for BF16); the largest difference is printed."""
    nx, ny, phi0, p = _case(wall)
    p["form"] = form
    out = [_gpu(pf, nx, ny, wall, p, phi0, 60, st, storage).populations() for st in ("gather", march)]
    worst = 0.0
    for a, b in zip(out[0], out[1]):
        scale = float(np.abs(a).max())
        diff = float(np.abs(a.astype(np.float64) - b).max())
        worst = max(worst, diff / scale)
    print(f"MARCH=GATHER {form} {storage} walls={wall}: largest difference / scale {worst:.2e}")
    assert worst <= {"fp32": 2e-5, "fp16": 2e-3, "bf16": 1e-2}[storage], worst


@pytest.mark.parametrize("wall", [False, True])
@pytest.mark.parametrize("storage,tol_phi,tol_u", [("fp16", 2e-4, 2e-5), ("bf16", 2e-3, 2e-4)])
def test_march_16bit_against_oracle(pf, orc, storage, tol_phi, tol_u, wall):
    nx, ny, phi0, p = _case(wall)
    p["form"] = "STF1"
    d = _gpu(pf, nx, ny, wall, p, phi0, 200, "march", storage)
    e_phi, e_u = _errs(d.fields(), _oracle(orc, nx, ny, wall, p, phi0, 200))
    assert e_phi <= tol_phi and e_u <= tol_u, (e_phi, e_u)


@pytest.mark.parametrize("shape,wall", [((192, 100), False), ((64, 600), True), ((320, 44), True),
                                        ((48, 8), False)])
def test_march_work_split(pf, shape, wall, march="march"):
    """CTA shares that start and end inside strips and span strip boundaries
    (several segments per CTA), a one-strip lattice narrower than the strip,
    the smallest height the mode accepts: equal to the gather mode."""
    nx, ny = shape
    phi0 = wl.smooth_random(nx, ny, seed=nx + ny, amp=0.7)
    p = dict(sigma=0.01, W=4.0, M=0.1, rho1=1.0, rho2=0.5, nu1=0.1, nu2=0.1, form="CSF1",
             uw_top=0.01 if wall else 0.0, gy=-1e-5)
    a = _gpu(pf, nx, ny, wall, p, phi0, 40, "gather").populations()
    b = _gpu(pf, nx, ny, wall, p, phi0, 40, march).populations()
    for x, y in zip(a, b):
        assert float(np.abs(x.astype(np.float64) - y).max()) <= 2e-5 * float(np.abs(x).max())


def test_march_graphs_equal_plain_launches(pf):
    nx, ny, phi0, p = _case(True)
    p["form"] = "CSF1"
    a = _gpu(pf, nx, ny, True, p, phi0, 73, "march").populations()
    b = _gpu(pf, nx, ny, True, p, phi0, 73, "march", graphs=True).populations()
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_march_autotune_keeps_state(pf):
    nx, ny, phi0, p = _case(False)
    p["form"] = "STF1"
    d = _gpu(pf, nx, ny, False, p, phi0, 10, "gather")
    before = d.populations()
    mode = d.autotune(3)
    assert mode in ("gather", "boxes", "march", "gather8")
    for x, y in zip(before, d.populations()):
        np.testing.assert_array_equal(x, y)


def test_march_refusals(pf):
    with pytest.raises(pf.PflbmError):
        pf.Domain(64, 32, wall_y=True, wall_x=True).stage_mode("march")
    with pytest.raises(pf.PflbmError):
        pf.Domain(66, 32).stage_mode("march")         # nx not a multiple of 4
    with pytest.raises(pf.PflbmError):
        pf.Domain(68, 32, storage="fp16").stage_mode("march")  # 16-bit: multiple of 8
    with pytest.raises(pf.PflbmError):
        pf.Domain(64, 6).stage_mode("march")          # fewer than 8 rows
    pf.Domain(72, 8, storage="bf16").stage_mode("march")

"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on
the same seeded inputs.

Bar (plain FP32 step): after 1000 steps of the stationary-drop workload,
max |phi_gpu - phi_oracle| <= 1e-5 and max |u_gpu - u_oracle| <= 1e-6 for
every force form.  The same bar applies to the other cases below (walls
with moving plates, gravity and density contrast on ragged grids that leave
partial tiles, grids smaller than one tile).
"""
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


def run_pair(pf, orc, nx, ny, wall, params, phi0, steps, storage="fp32", graphs=False):
    d = pf.Domain(nx, ny, wall_y=wall, storage=storage)
    d.set_params(**params)
    d.init_phi(phi0.astype(np.float32))
    if graphs:
        d.graphs(True)
    d.step(steps)
    g = d.fields()
    # the oracle starts from the same float32 phi0 the GPU received
    s = orc.Sim(nx, ny, wall, orc.Params(**params), phi0.astype(np.float32).astype(np.float64))
    s.step(steps)
    o = s.macro()
    return d, g, s, o


def err(g, o, k):
    return float(np.abs(g[k].astype(np.float64) - o[k]).max())


@pytest.mark.parametrize("form", FORMS)
def test_stationary_drop_1000_steps(pf, orc, form):
    c = wl.stationary_drop(form)
    _, g, _, o = run_pair(pf, orc, c.nx, c.ny, False, c.params, c.phi0, 1000)
    e_phi, e_ux, e_uy = err(g, o, "phi"), err(g, o, "ux"), err(g, o, "uy")
    assert e_phi <= TOL_PHI and e_ux <= TOL_U and e_uy <= TOL_U, (e_phi, e_ux, e_uy)


@pytest.mark.parametrize("form", FORMS)
def test_walls_ragged_tiles(pf, orc, form):
    """37 x 29 (partial tiles in x and y), walls moving at -/+0.01, gravity,
    density ratio 4, viscosity ratio 2, drop off-centre."""
    nx, ny = 37, 29
    phi0 = wl.drop(nx, ny, 8.0, 4.0, xc=15.3, yc=13.1, periodic_y=False)
    p = dict(sigma=0.01, W=4.0, M=0.1, rho1=1.0, rho2=0.25, nu1=0.1, nu2=0.2,
             gy=-1e-5, uw_bottom=-0.01, uw_top=0.01, form=form)
    _, g, _, o = run_pair(pf, orc, nx, ny, True, p, phi0, 300)
    e = (err(g, o, "phi"), err(g, o, "ux"), err(g, o, "uy"))
    assert e[0] <= TOL_PHI and max(e[1:]) <= TOL_U, e


@pytest.mark.parametrize("shape,wall", [((4, 4), False), ((5, 7), True), ((6, 33), False)])
def test_tiny_grids(pf, orc, shape, wall):
    nx, ny = shape
    phi0 = wl.smooth_random(nx, ny, seed=nx * ny, amp=0.8)
    p = dict(sigma=0.01, W=4.0, M=0.1, rho1=1.0, rho2=0.5, nu1=0.1, nu2=0.1, form="CSF2",
             uw_top=0.01 if wall else 0.0)
    _, g, _, o = run_pair(pf, orc, nx, ny, wall, p, phi0, 50)
    assert err(g, o, "phi") <= TOL_PHI and max(err(g, o, "ux"), err(g, o, "uy")) <= TOL_U


@pytest.mark.parametrize("form", FORMS)
def test_all_fields_one_step(pf, orc, form):
    """Every read-back field after a few steps from a non-equilibrium field
    (chemical potential, both pressures, force).  Tolerance: float32 state
    rounding (unit 6e-8 on h_0 ~ phi ~ 1) reaches derived fields through
    differences of O(1) values (grad phi, mu = 4 beta phi^3 - ... - kappa lap
    phi, P = sum f); 1e-4 of each field's scale plus 1e-8 absolute bounds it
    with margin (about 1000 ulps)."""
    nx, ny = 48, 40
    phi0 = wl.smooth_random(nx, ny, seed=3, amp=0.9)
    p = dict(sigma=0.02, W=4.0, M=0.1, rho1=1.0, rho2=0.5, nu1=0.1, nu2=0.05, gx=1e-5,
             form=form)
    _, g, _, o = run_pair(pf, orc, nx, ny, False, p, phi0, 3)
    for k in ("phi", "rho", "ux", "uy", "P", "mu", "p_h", "Fx", "Fy"):
        scale = max(1e-6, float(np.abs(o[k]).max()))
        assert err(g, o, k) <= 1e-4 * scale + 1e-8, (k, err(g, o, k), scale)


@pytest.mark.parametrize("wall", [False, True])
def test_initial_populations(pf, orc, wall):
    nx, ny = 40, 24
    phi0 = wl.drop(nx, ny, 7.0, 4.0, periodic_y=not wall)
    p = dict(sigma=0.01, W=4.0, M=0.1, form="STF1")
    d = pf.Domain(nx, ny, wall_y=wall).set_params(**p).init_phi(phi0.astype(np.float32))
    f, h = d.populations()
    s = orc.Sim(nx, ny, wall, orc.Params(**p), phi0.astype(np.float32).astype(np.float64))
    assert np.abs(f).max() == 0.0
    assert np.abs(h - s.h).max() < 1e-7


def test_populations_after_steps(pf, orc):
    nx, ny = 40, 24
    phi0 = wl.drop(nx, ny, 7.0, 4.0, periodic_y=False)
    p = dict(sigma=0.01, W=4.0, M=0.1, rho2=0.5, uw_top=0.01, form="CPF2")
    d, g, s, o = run_pair(pf, orc, nx, ny, True, p, phi0, 20)
    f, h = d.populations()
    assert np.abs(f - s.f).max() < 1e-7
    assert np.abs(h - s.h).max() < 1e-6


def test_deterministic_and_graph_equal(pf):
    c = wl.stationary_drop("CSF1")
    outs = []
    for graphs in (False, False, True):
        d = pf.Domain(c.nx, c.ny).set_params(**c.params).init_phi(c.phi0.astype(np.float32))
        d.graphs(graphs)
        d.step(200)
        f, h = d.populations()
        outs.append((f, h))
    for f, h in outs[1:]:
        np.testing.assert_array_equal(f, outs[0][0])
        np.testing.assert_array_equal(h, outs[0][1])


def test_checkpoint_resume_keeps_the_default_rho0(pf):
    """With gravity, F_g = (rho - rho0) g depends on rho0, which by default
    is the mean density of phi0: the blob carries it, so a resumed run
    continues bitwise even though the resuming domain never saw phi0."""
    nx, ny = 64, 48
    phi0 = wl.bubble(nx, ny, 10.0, 4.0).astype(np.float32)
    p = dict(sigma=0.01, W=4.0, M=0.1, rho1=1.0, rho2=0.2, nu1=0.1, nu2=0.1, gy=-1e-5)
    a = pf.Domain(nx, ny, wall_y=True).set_params(**p).init_phi(phi0)
    a.step(30)
    blob = a.save_state()
    a.step(40)
    b = pf.Domain(nx, ny, wall_y=True).set_params(**p).load_state(blob)
    b.step(40)
    for x, y in zip(a.populations(), b.populations()):
        np.testing.assert_array_equal(x, y)
    # parameters set again after the resume keep the run's rho0 as well
    b.set_params(**p)
    a.set_params(**p)
    a.step(5)
    b.step(5)
    for x, y in zip(a.populations(), b.populations()):
        np.testing.assert_array_equal(x, y)


def test_checkpoint_resume_bitwise(pf):
    c = wl.stationary_drop("PF2")
    a = pf.Domain(c.nx, c.ny).set_params(**c.params).init_phi(c.phi0.astype(np.float32))
    a.step(100)
    blob = a.save_state()
    a.step(50)
    b = pf.Domain(c.nx, c.ny).set_params(**c.params)
    b.load_state(blob)
    assert b.t == 100
    b.step(50)
    for x, y in zip(a.populations(), b.populations()):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("form", ["STF1", "CSF2"])
def test_diagnostics_match_oracle(pf, orc, form):
    c = wl.stationary_drop(form)
    d, g, s, o = run_pair(pf, orc, c.nx, c.ny, False, c.params, c.phi0, 500)
    dg = d.diagnostics(32.0, 32.0, 8.0, 16.0 + 12.0)
    lo = orc.laplace(o, 32, 32, 16.0, 4.0)
    assert dg["status"] == "PFLBM_OK"
    assert abs(dg["mass"] - o["phi"].sum()) < 1e-3
    assert abs(dg["umax"] - orc.umax(o)) < 1e-6
    assert abs(dg["R_num"] - lo["R_num"]) < 1e-5
    assert abs(dg["dp"] - lo["dp"]) < 1e-6
    assert abs(dg["taylor_D"] - orc.taylor_D(o)) < 1e-5
    assert abs(dg["xc1"] - orc.mass_centre_x(o)) < 1e-4


def test_mass_conserved_on_gpu(pf):
    """sum phi drifts only by float32 rounding over 2000 steps."""
    c = wl.stationary_drop("STF2")
    d = pf.Domain(c.nx, c.ny).set_params(**c.params).init_phi(c.phi0.astype(np.float32))
    m0 = d.diagnostics()["mass"]
    d.step(2000)
    m1 = d.diagnostics()["mass"]
    assert abs(m1 - m0) < 1e-3


def test_nonfinite_state_is_reported(pf):
    """A NaN in the initial field (host-side input) surfaces as EUNSTABLE."""
    c = wl.stationary_drop("STF1")
    phi0 = c.phi0.astype(np.float32).copy()
    phi0[5, 5] = np.nan
    d = pf.Domain(c.nx, c.ny).set_params(**{**c.params, "rho0": 1.0}).init_phi(phi0)
    d.step(3)
    dg = d.diagnostics()
    assert dg["status"] == "PFLBM_EUNSTABLE" and dg["nonfinite"] > 0

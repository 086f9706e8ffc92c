"""Oracle pin: the whole composition of a step against a second transcription.

The moment, stencil and invariant pins fix the oracle's pieces; this test
fixes how they are put together (pass order, the time level of d_t(phi u),
which u enters div(phi u), the wall and side-wall ghosts, the bounce-back
terms, the order of collision and streaming).  ``bruteforce_step`` is written
straight from Sec. 3 (Eqs. fh, eq, heq_CH, P_LBM, CH_LB_force, mac, ICS-1st,
ICS-sec), Sec. 2.2 (the eight force forms) and Sec. 4 (Ladd's bounce-back),
as scalar Python loops that share nothing with the oracle.  Both advance the
same random state of a few nodes (non-zero velocity, a density contrast,
gravity, moving walls) by 1, 2 and 3 steps and must agree to 1e-13.
"""
import numpy as np
import pytest

import bruteforce_step as bf

FORMS = ("STF1", "STF2", "CPF1", "CPF2", "PF1", "PF2", "CSF1", "CSF2")
W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)

CASES = {
    # name: (nx, ny, wall_y, wall_x, gx, gy, uw_bottom, uw_top)
    "periodic_4x4": (4, 4, False, False, 2e-3, -3e-3, 0.0, 0.0),
    "walls_4x5": (4, 5, True, False, 1e-3, -4e-3, -0.01, 0.015),
    "walls_5x4": (5, 4, True, False, 0.0, -2e-3, 0.02, 0.0),
    "side_walls_4x5": (4, 5, True, True, 0.0, -3e-3, 0.0, 0.0),
    "side_walls_periodic_y_5x4": (5, 4, False, True, 0.0, 2e-3, 0.0, 0.0),
}


def _state(nx, ny, seed):
    """A random state: phi of a few Fourier modes plus noise, populations near
    their weights with noise (non-zero momentum and pressure), and a random
    (phi u)^{t-1}."""
    rng = np.random.default_rng(seed)
    Y, X = np.mgrid[0:ny, 0:nx].astype(float)
    phi = 0.6 * np.sin(2 * np.pi * X / nx + rng.uniform(0, 6)) * np.cos(2 * np.pi * Y / ny + rng.uniform(0, 6))
    phi += 0.15 * rng.uniform(-1, 1, (ny, nx))
    h = W[:, None, None] * (phi[None] + 0.05 * rng.uniform(-1, 1, (9, ny, nx)))
    f = W[:, None, None] * (0.02 + 0.06 * rng.uniform(-1, 1, (9, ny, nx)))
    q = 0.01 * rng.uniform(-1, 1, (2, ny, nx))
    return f, h, q


def _params(form, gx, gy, uwb, uwt):
    return dict(sigma=0.02, W=2.5, M=0.05, tau_h=0.9, rho1=1.0, rho2=0.3, nu1=0.1, nu2=0.04,
                gx=gx, gy=gy, rho0=0.7, uw_bottom=uwb, uw_top=uwt, eps=1e-6, form=form)


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("first", [False, True])
def test_oracle_equals_bruteforce(orc, case, form, first):
    nx, ny, wall_y, wall_x, gx, gy, uwb, uwt = CASES[case]
    par = _params(form, gx, gy, uwb, uwt)
    f, h, q = _state(nx, ny, seed=FORMS.index(form) + 17 * len(case))
    sim = orc.Sim(nx, ny, wall_y, orc.Params(**par), np.zeros((ny, nx)), wall_x=wall_x)
    sim.f[...] = f
    sim.h[...] = h
    sim.phiu_prev[...] = q
    sim.t = 0 if first else 1
    lat = bf.Lattice(nx, ny, wall_y, wall_x)
    bstate = (f.tolist(), h.tolist(), q.tolist())
    for k in range(3):
        sim.step(1)
        bstate = bf.step(lat, par, *bstate, first and k == 0)
        for name, a, b in (("f", sim.f, bstate[0]), ("h", sim.h, bstate[1]),
                           ("phi u", sim.phiu_prev, bstate[2])):
            err = float(np.abs(a - np.array(b)).max())
            assert err < 1e-13, (case, form, k + 1, name, err)

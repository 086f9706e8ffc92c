"""Oracle pins: per-node pieces of the scheme against the moment conditions the
Chapman-Enskog recovery of Sec. 3 requires (Eqs. fh, heq_CH, P_LBM,
CH_LB_force, mac).  These conditions are consequences of the paper's macroscopic
equations, not retypes of the oracle's formulas: a dropped term, wrong weight,
wrong sign or transposed index in f^eq, h^eq, F_i or H_i breaks one of them.
"""
import numpy as np
import pytest

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=float)
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=float)
CS2 = 1.0 / 3.0

rng = np.random.default_rng(1234)
CASES = [tuple(rng.uniform(-1, 1, 6)) for _ in range(20)]


def mom(a):
    """zeroth, first, second moments of a 9-vector"""
    m0 = a.sum()
    m1 = np.array([(a * CX).sum(), (a * CY).sum()])
    m2 = np.array([[(a * CX * CX).sum(), (a * CX * CY).sum()],
                   [(a * CY * CX).sum(), (a * CY * CY).sum()]])
    return m0, m1, m2


@pytest.mark.parametrize("c", CASES)
def test_feq_moments(orc, c):
    """sum f^eq = P, sum c f^eq = cs^2 rho u, sum cc f^eq = cs^2 P I + cs^2 rho uu
    (pressure-based distribution of He et al., Sec. 3)."""
    P, rho, ux, uy = c[0] * 1e-2, 1.0 + 0.5 * c[1], 0.05 * c[2], 0.05 * c[3]
    m0, m1, m2 = mom(orc.feq(P, rho, ux, uy))
    u = np.array([ux, uy])
    assert m0 == pytest.approx(P, abs=1e-15)
    np.testing.assert_allclose(m1, CS2 * rho * u, atol=1e-15)
    np.testing.assert_allclose(m2, CS2 * P * np.eye(2) + CS2 * rho * np.outer(u, u), atol=1e-15)


@pytest.mark.parametrize("c", CASES)
def test_heq_moments(orc, c):
    """sum h^eq = phi, sum c h^eq = phi u, sum cc h^eq = cs^2 eta mu I (Eq. heq_CH)."""
    phi, mu, eta, ux, uy = c[0], 1e-3 * c[1], 3.0 * abs(c[2]) + 0.1, 0.05 * c[3], 0.05 * c[4]
    m0, m1, m2 = mom(orc.heq(phi, mu, eta, ux, uy))
    assert m0 == pytest.approx(phi, abs=1e-15)
    np.testing.assert_allclose(m1, [phi * ux, phi * uy], atol=1e-15)
    np.testing.assert_allclose(m2, CS2 * eta * mu * np.eye(2), atol=1e-15)


@pytest.mark.parametrize("c", CASES)
def test_force_moments(orc, c):
    """sum F_i = u . grad(cs^2 rho) and sum c F_i = cs^2 F: the two relations the
    macroscopic P and u of Eq. mac rely on.  They fix the reading
    Gamma_i = w_i (1 + s_i) with grad-rho weight w_i s_i (Eq. P_LBM)."""
    ux, uy = 0.05 * c[0], 0.05 * c[1]
    Fx, Fy, drx, dry = 1e-3 * c[2], 1e-3 * c[3], 0.3 * c[4], 0.3 * c[5]
    m0, m1, _ = mom(orc.fforce(ux, uy, Fx, Fy, drx, dry))
    assert m0 == pytest.approx(CS2 * (ux * drx + uy * dry), abs=1e-16)
    np.testing.assert_allclose(m1, [CS2 * Fx, CS2 * Fy], atol=1e-16)


def test_force_literal_reading_fails_moments(orc):
    """The literal printed Gamma_i = w_i + s_i does not give sum c F_i = cs^2 F;
    shown here with plain numpy so the chosen reading is justified by a test."""
    ux, uy, Fx, Fy = 0.03, -0.02, 1e-3, 2e-3
    W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    cu = CX * ux + CY * uy
    s = 3 * cu + 4.5 * cu ** 2 - 1.5 * (ux * ux + uy * uy)
    gam = W + s
    Fi = (CX - ux) * gam * Fx + (CY - uy) * gam * Fy
    assert abs((Fi * CX).sum() - CS2 * Fx) > 1e-5


@pytest.mark.parametrize("c", CASES)
@pytest.mark.parametrize("tau_h", [0.8, 1.0, 0.5 + 3 ** 0.5 / 6, 1.7])
def test_hsource_moments(orc, c, tau_h):
    """sum H_i = 0, sum c H_i = d_t(phi u), sum cc H_i = cs^2 A I with
    A = 3 tau2/(tau_h tau1) div(phi u) (Eq. CH_LB_force, wbar conditions)."""
    div, dtx, dty = 1e-3 * c[0], 1e-3 * c[1], 1e-3 * c[2]
    m0, m1, m2 = mom(orc.hsource(tau_h, div, dtx, dty))
    t1 = tau_h - 0.5
    t2 = tau_h * tau_h - tau_h + 1 / 6
    A = 3 * t2 / (tau_h * t1) * div
    assert m0 == pytest.approx(0.0, abs=1e-17)
    np.testing.assert_allclose(m1, [dtx, dty], atol=1e-17)
    np.testing.assert_allclose(m2, CS2 * A * np.eye(2), atol=1e-17)


def test_hsource_liang_special_case(orc):
    """tau_h = 1/2 + sqrt(3)/6 gives tau2 = 0: the div(phi u) term vanishes and
    the scheme reduces to Liang et al. (Sec. 3)."""
    out = orc.hsource(0.5 + 3 ** 0.5 / 6, 1.0, 0.0, 0.0)
    np.testing.assert_allclose(out, 0.0, atol=1e-15)


def test_equilibria_at_rest(orc):
    """At rest (u = 0, P = 0) f^eq vanishes and h^eq has only the mu terms."""
    np.testing.assert_array_equal(orc.feq(0.0, 1.3, 0.0, 0.0), np.zeros(9))
    h = orc.heq(0.7, 0.0, 6.0, 0.0, 0.0)
    np.testing.assert_array_equal(h, [0.7] + [0.0] * 8)

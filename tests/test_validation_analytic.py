"""Pins of the capillary-wave analytic solution (Sec. 5.3) against facts
other than its own formula."""
import math

import numpy as np
import pytest

from paper_2012_14729_gb300 import validation as v


def test_roots_solve_the_quartic():
    z, beta, w02, a = v.prosperetti_roots(0.02, 2 * math.pi / 80, 0.0125, 1.0, 0.5)
    for zi in z:
        p = zi ** 4 - 4 * beta * math.sqrt(a) * zi ** 3 + 2 * (1 - 6 * beta) * a * zi ** 2 + \
            4 * (1 - 3 * beta) * a ** 1.5 * zi + (1 - 4 * beta) * a * a + w02
        assert abs(p) <= 1e-12 * max(1.0, abs(zi) ** 4)


def test_initial_amplitude_is_h0():
    for rho2 in (1.0, 0.1):
        h = v.prosperetti_amplitude([0.0], 0.02, 2 * math.pi / 80, 0.0125, 1.0, rho2)
        assert h[0] == pytest.approx(1.0, abs=1e-10)


def test_inviscid_limit_is_a_standing_wave():
    """nu -> 0: h(t) / h0 -> cos(omega_0 t), omega_0^2 = sigma k^3 / (rho1 + rho2)."""
    k, sigma = 2 * math.pi / 80, 0.0125
    w0 = math.sqrt(sigma * k ** 3 / 2.0)
    t = np.linspace(0, 3 * 2 * math.pi / w0, 50)
    h = v.prosperetti_amplitude(t, 1e-9, k, sigma, 1.0, 1.0)
    np.testing.assert_allclose(h, np.cos(w0 * t), atol=2e-3)


def test_free_surface_limit_has_lambs_damping_rate():
    """rho2 = 0 (beta = 0, a free surface) with small viscosity: the wave
    envelope decays like exp(-2 nu k^2 t), Lamb's classical rate."""
    k, sigma, nu = 2 * math.pi / 80, 0.0125, 2e-4
    w0 = math.sqrt(sigma * k ** 3 / 1.0)
    T = 2 * math.pi / w0
    env = []
    for m in (10, 20):
        t = np.linspace(m * T, (m + 1) * T, 400)
        env.append(np.abs(v.prosperetti_amplitude(t, nu, k, sigma, 1.0, 0.0)).max())
    rate = -math.log(env[1] / env[0]) / (10 * T)
    assert rate == pytest.approx(2 * nu * k * k, rel=0.03)


def test_overdamped_wave_does_not_oscillate():
    """nu k^2 >> omega_0: the amplitude decays monotonically and stays
    positive."""
    k, sigma = 2 * math.pi / 80, 1e-5
    h = v.prosperetti_amplitude(np.linspace(0, 2e5, 200), 0.5, k, sigma, 1.0, 1.0)
    assert np.all(np.diff(h) <= 1e-12) and np.all(h > 0)


def test_interface_height_and_error():
    ny, nx = 240, 80
    y = np.arange(ny)[:, None]
    x = np.arange(nx)[None, :]
    yi = 120.3 + 1.6 * np.cos(2 * math.pi * x / nx)
    phi = np.tanh(2 * (yi - y) / 4.0)
    assert v.interface_height(phi, 0) == pytest.approx(121.9, abs=0.05)
    assert v.wave_amplitude(phi) == pytest.approx(1.6, abs=0.05)



def test_time_averaged_error_is_the_rms_over_the_window():
    """Eq. capilary_error: sqrt of the time average of the squared difference.
    Closed forms: a constant offset d gives |d|; a sine difference over whole
    periods gives amplitude / sqrt 2; a linear drift a t over [0, T] gives
    a T / sqrt 3 (trapezoid error O(dt^2))."""
    t = np.linspace(0.0, 10.0, 2001)
    h = np.cos(t)
    assert v.time_averaged_error(t, h, h) == 0.0
    assert v.time_averaged_error(t, h + 0.3, h) == pytest.approx(0.3, rel=1e-12)
    T = 4 * np.pi
    t2 = np.linspace(0.0, T, 4001)
    assert v.time_averaged_error(t2, 0.2 * np.sin(t2), 0 * t2) == pytest.approx(0.2 / math.sqrt(2),
                                                                              rel=1e-6)
    assert v.time_averaged_error(t2, 0.01 * t2, 0 * t2) == pytest.approx(0.01 * T / math.sqrt(3),
                                                                       rel=1e-6)


def test_error_window_is_25_over_omega0():
    from paper_2012_14729_gb300 import workloads as wl
    c = wl.capillary_wave("STF1", H=80)
    w0 = v.omega0(c.meta["k"], c.params["sigma"], c.params["rho1"], c.params["rho2"])
    # omega_0^2 = sigma k^3 / (rho1 + rho2)
    assert w0 ** 2 == pytest.approx(c.params["sigma"] * (2 * math.pi / 80) ** 3 / 2.0)
    n = v.error_window_steps(c, 90)
    assert n % 90 == 0 and 25 / w0 <= n < 25 / w0 + 90

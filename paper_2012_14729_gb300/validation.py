"""Capillary-wave validation (Sec. 5.3): the analytic amplitude of a small
interface wave between two viscous fluids of equal kinematic viscosity
(Prosperetti's initial-value solution, Eq. capillary_wave) and the
measurement of the simulated amplitude.

The analytic solution is host-side reference mathematics for checking the
CUDA path, not a step of the method.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special


def prosperetti_roots(nu: float, k: float, sigma: float, rho1: float, rho2: float):
    """The four roots z_i of the quartic of Eq. error_function and
    (beta, omega_0^2, nu k^2) of Sec. 5.3."""
    beta = rho1 * rho2 / (rho1 + rho2) ** 2
    w02 = sigma * k ** 3 / (rho1 + rho2)
    a = nu * k * k
    coeffs = [1.0, -4.0 * beta * math.sqrt(a), 2.0 * (1.0 - 6.0 * beta) * a,
              4.0 * (1.0 - 3.0 * beta) * a ** 1.5, (1.0 - 4.0 * beta) * a * a + w02]
    return np.roots(coeffs).astype(complex), beta, w02, a


def prosperetti_amplitude(t, nu: float, k: float, sigma: float, rho1: float, rho2: float):
    """h(t) / h0 of Eq. capillary_wave at times t (array).  The products
    exp((z_i^2 - nu k^2) t) erfc(z_i sqrt t) are evaluated as
    exp(-nu k^2 t) w(i z_i sqrt t), w the Faddeeva function, which stays
    finite for every t."""
    t = np.asarray(t, dtype=float)
    z, beta, w02, a = prosperetti_roots(nu, k, sigma, rho1, rho2)
    out = 4.0 * (1.0 - 4.0 * beta) * a * a / (8.0 * (1.0 - 4.0 * beta) * a * a + w02) * \
        special.erfc(np.sqrt(a * t))
    s = np.zeros(t.shape, dtype=complex)
    for i in range(4):
        Zi = np.prod([z[j] - z[i] for j in range(4) if j != i])
        s += z[i] / Zi * w02 / (z[i] ** 2 - a) * np.exp(-a * t) * \
            special.wofz(1j * z[i] * np.sqrt(t))
    return out + s.real


def interface_height(phi: np.ndarray, x: int) -> float:
    """Height of the phi = 0 level in column x (phi > 0 below it), by linear
    interpolation between the two nodes that bracket the sign change."""
    col = phi[:, x]
    idx = np.nonzero((col[:-1] > 0) & (col[1:] <= 0))[0]
    if len(idx) == 0:
        return math.nan
    j = idx[0]
    return j + col[j] / (col[j] - col[j + 1])


def wave_amplitude(phi: np.ndarray) -> float:
    """Amplitude of the cos(k x) wave: half the height difference between
    the crest column x = 0 and the trough column x = nx / 2."""
    nx = phi.shape[1]
    return 0.5 * (interface_height(phi, 0) - interface_height(phi, nx // 2))


def omega0(k: float, sigma: float, rho1: float, rho2: float) -> float:
    """Inviscid capillary frequency, omega_0^2 = sigma k^3 / (rho1 + rho2)."""
    return math.sqrt(sigma * k ** 3 / (rho1 + rho2))


def time_averaged_error(t, h_num, h_th) -> float:
    """E_2 of Eq. capilary_error: the root of the time average of
    |h(t)/h0 - h_exact(t)/h0|^2 over the sampled window [t_0, t_end] (the
    paper's window is [0, 25 / omega_0]), the integral taken by the
    trapezoidal rule over the samples."""
    t = np.asarray(t, float)
    d2 = (np.asarray(h_num, float) - np.asarray(h_th, float)) ** 2
    integral = float(np.sum(0.5 * (d2[1:] + d2[:-1]) * np.diff(t)))
    return math.sqrt(integral / (t[-1] - t[0]))


def error_window_steps(case, every: int) -> int:
    """Steps covering the paper's error window [0, 25 / omega_0], rounded up
    to a multiple of `every`."""
    p = case.params
    t_end = 25.0 / omega0(case.meta["k"], p["sigma"], p["rho1"], p["rho2"])
    return int(math.ceil(t_end / every)) * every


def run_capillary_wave(pflbm, case, every: int, steps=None):
    """Advance a capillary-wave case on the GPU (module `pflbm`, the CUDA
    binding), sampling the amplitude every `every` steps over `steps` steps
    (default: the error window [0, 25 / omega_0]); returns the sample times,
    h_num / h0, the analytic h / h0 and E_2."""
    if steps is None:
        steps = error_window_steps(case, every)
    p = case.params
    d = pflbm.Domain(case.nx, case.ny, wall_y=True).set_params(**p)
    d.init_phi(case.phi0.astype(np.float32))
    h0 = case.meta["h0"]
    ts, hs = [], []
    for n in range(0, steps + 1, every):
        if n:
            d.step(every)
        ts.append(n)
        hs.append(wave_amplitude(d.read("phi")) / h0)
    ts = np.asarray(ts, float)
    th = prosperetti_amplitude(ts, p["nu1"], case.meta["k"], p["sigma"], p["rho1"], p["rho2"])
    return ts, np.asarray(hs), th, time_averaged_error(ts, hs, th)

"""Seeded synthetic inputs shaped like the paper's benchmarks (Sec. 5).

This module holds no arithmetic of the lattice Boltzmann method: it only
builds initial order-parameter fields phi0 (and the small random numbers some
workloads add) that the CUDA path and the FP64 oracle both start from.  Phases
follow the paper's convention phi = +1 in fluid 1 and phi = -1 in fluid 2.

Profiles (all tanh of width W, Sec. 2.1 equilibrium profile):
  drop          phi = tanh(2 (R - r)/W)                       stationary drop, Sec. 5.1
  two_drops     phi = 1 + tanh(..R1..) + tanh(..R2..)           merging drops, Sec. 5.2
  wave          heavy fluid (phi = +1) below y = y0 + a sin(2 pi x / nx)   capillary wave, Sec. 5.3
  bubble        light bubble (phi = -1) of radius R in fluid 1  rising bubble, Sec. 5.4
  ellipse       drop with semi-axes R (1 + e), R (1 - e)        oscillating drop
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def _grid(nx: int, ny: int):
    x = np.arange(nx, dtype=np.float64)[None, :]
    y = np.arange(ny, dtype=np.float64)[:, None]
    return x, y


def _dist(nx, ny, xc, yc, periodic_x=True, periodic_y=True):
    x, y = _grid(nx, ny)
    dx = x - xc
    dy = y - yc
    if periodic_x:
        dx = dx - nx * np.round(dx / nx)
    if periodic_y:
        dy = dy - ny * np.round(dy / ny)
    return dx, dy


def drop(nx, ny, R, W, xc=None, yc=None, periodic_y=True):
    """Circular drop of fluid 1 (phi = +1 inside) centred at (xc, yc)."""
    xc = nx / 2 if xc is None else xc
    yc = ny / 2 if yc is None else yc
    dx, dy = _dist(nx, ny, xc, yc, True, periodic_y)
    r = np.sqrt(dx * dx + dy * dy)
    return np.tanh(2.0 * (R - r) / W)


def ellipse(nx, ny, R, W, e=0.1, xc=None, yc=None):
    """Drop with semi-axes R(1+e) along x and R(1-e) along y (signed distance
    approximated by the radial scaling of the ellipse)."""
    xc = nx / 2 if xc is None else xc
    yc = ny / 2 if yc is None else yc
    dx, dy = _dist(nx, ny, xc, yc)
    a, b = R * (1 + e), R * (1 - e)
    rho = np.sqrt((dx / a) ** 2 + (dy / b) ** 2)
    rm = math.sqrt(a * b)
    return np.tanh(2.0 * rm * (1.0 - rho) / W)


def two_drops(nx, ny, R1, R2, gap, W):
    """Two drops on the horizontal midline with `gap` cells between their
    rims, phi = 1 + tanh(drop 1) + tanh(drop 2) (-1 outside)."""
    x1 = nx / 2 - R1 - gap / 2
    x2 = nx / 2 + R2 + gap / 2
    yc = ny / 2
    d1x, d1y = _dist(nx, ny, x1, yc)
    d2x, d2y = _dist(nx, ny, x2, yc)
    r1 = np.sqrt(d1x ** 2 + d1y ** 2)
    r2 = np.sqrt(d2x ** 2 + d2y ** 2)
    return 1.0 + np.tanh(2.0 * (R1 - r1) / W) + np.tanh(2.0 * (R2 - r2) / W)


def wave(nx, ny, amp, W, y0=None):
    """Flat interface at y0 perturbed by amp sin(2 pi x / nx); heavy fluid 1
    (phi = +1) below, light fluid 2 above (walls at bottom and top)."""
    y0 = ny / 2 if y0 is None else y0
    x, y = _grid(nx, ny)
    yi = y0 + amp * np.sin(2.0 * math.pi * x / nx)
    return np.tanh(2.0 * (yi - y) / W)


def bubble(nx, ny, R, W, xc=None, yc=None):
    """Light bubble (phi = -1 inside) in fluid 1, walls at bottom and top."""
    xc = nx / 2 if xc is None else xc
    yc = ny / 4 if yc is None else yc
    dx, dy = _dist(nx, ny, xc, yc, True, False)
    r = np.sqrt(dx * dx + dy * dy)
    return -np.tanh(2.0 * (R - r) / W)


def noise(nx, ny, amp, seed=0):
    """Uniform noise in [-amp, amp] from a seeded host generator."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-amp, amp, size=(ny, nx))


def smooth_random(nx, ny, seed=0, modes=3, amp=0.5):
    """A smooth periodic random field (a few low Fourier modes) in (-1, 1)."""
    rng = np.random.default_rng(seed)
    x, y = _grid(nx, ny)
    out = np.zeros((ny, nx))
    for _ in range(modes):
        kx = rng.integers(1, 3)
        ky = rng.integers(1, 3)
        ph = rng.uniform(0, 2 * math.pi, 2)
        out += rng.uniform(-1, 1) * np.cos(2 * math.pi * kx * x / nx + ph[0]) * \
            np.cos(2 * math.pi * ky * y / ny + ph[1])
    return amp * out / max(1.0, np.abs(out).max())


# ---------------------------------------------------------------------------
# named workloads
# ---------------------------------------------------------------------------

@dataclass
class Case:
    """One run: grid, walls, parameters (lattice units) and phi0."""
    name: str
    nx: int
    ny: int
    wall_y: bool
    params: dict
    phi0: np.ndarray = field(repr=False)
    steps: int = 0
    meta: dict = field(default_factory=dict)


def stationary_drop(form="STF1", n=64, R=16.0, W=4.0, sigma=0.01, M=0.1, nu=0.1,
                    tau_h=1.0):
    """64x64 periodic, drop R = 16 at the centre, W = 4, rho1 = rho2 = 1,
    nu = 0.1, M = 0.1, sigma = 0.01, g = 0 (stationary drop, Sec. 5.1)."""
    p = dict(sigma=sigma, W=W, M=M, tau_h=tau_h, rho1=1.0, rho2=1.0, nu1=nu,
             nu2=nu, form=form)
    return Case("stationary_drop", n, n, False, p, drop(n, n, R, W), 5000,
                {"R": R, "xc": n / 2, "yc": n / 2})


def merging_drops(form="STF1", nx=256, ny=128, R=25.0, gap=2.0, W=5.0,
                  ratio=5.0, visc_ratio=1.0, sigma=1e-3, M=0.05, nu1=0.1):
    """256x128 periodic, two R = 25 drops 52 apart (2-cell gap), W = 5,
    rho1/rho2 = ratio, nu1/nu2 = visc_ratio, sigma = 1e-3, M = 0.05 (Sec. 5.2).

    Defaults are the paper's own merging-drop ratios (rho_d/rho_s = 5, equal
    kinematic viscosities); the stated rho1/rho2 = 1000, nu1/nu2 = 10
    (ratio=1000, visc_ratio=10) diverges within the first thousand steps with
    this scheme."""
    p = dict(sigma=sigma, W=W, M=M, tau_h=1.0, rho1=1.0, rho2=1.0 / ratio,
             nu1=nu1, nu2=nu1 / visc_ratio, form=form)
    return Case("merging_drops", nx, ny, False, p, two_drops(nx, ny, R, R, gap, W),
                20000, {"R": R})


def capillary_bubble(kind="bubble", form="STF1", nx=512, ny=1024, W=5.0,
                     ratio=10.0, nu1=0.1, visc_ratio=1.0, sigma=1e-3, M=0.05,
                     g=1e-6, R=64.0, seed=0, noise_amp=1e-3):
    """512x1024, walls at bottom and top, periodic sides.  'wave': flat
    interface at ny/2 perturbed by 0.01 nx sin(2 pi x/nx), g = 0; 'bubble':
    R = 64 light bubble at (nx/2, ny/4) under gravity g (along -y).  Both with
    seeded uniform noise of amplitude noise_amp on phi0 (Secs. 5.3, 5.4).

    Defaults are the stable fallback rho1/rho2 = 10 with equal kinematic
    viscosities (dynamic-viscosity ratio 10), the largest ratios the paper
    runs (Sec. 5.4); the stated rho1/rho2 = 1000, nu1/nu2 = 100 (pass
    ratio=1000, nu1=1.0, visc_ratio=100) diverges within 20 steps with this
    scheme, in the oracle as on the GPU."""
    if kind == "wave":
        phi0 = wave(nx, ny, 0.01 * nx, W)
        gy = 0.0
    else:
        phi0 = bubble(nx, ny, R, W)
        gy = -g
    phi0 = np.clip(phi0 + noise(nx, ny, noise_amp, seed), -1.0, 1.0)
    p = dict(sigma=sigma, W=W, M=M, tau_h=1.0, rho1=1.0, rho2=1.0 / ratio,
             nu1=nu1, nu2=nu1 / visc_ratio, gx=0.0, gy=gy, form=form)
    meta = {"R": R} if kind == "wave" else {"R": R, "xc": nx / 2, "yc": ny / 4}
    return Case(f"capillary_{kind}", nx, ny, True, p, phi0, 50000, meta)


UG_PHYS = math.sqrt(2 * 0.25 * 0.98)  # reference velocity sqrt(2 R g) of Sec. 5.4, m/s


def rising_bubble(form="STF1", nx=120, Ug=0.01, W=8.0, M=0.05, tau_h=0.8, Re=35.0, Eo=10.0,
                  rho_ratio=10.0, mu_ratio=10.0):
    """The rising bubble of Sec. 5.4 on an nx x 2nx lattice: the paper's
    1 m x 2 m box (node spacing 1/nx m, walls half a spacing beyond the
    outer nodes), no-slip walls at bottom and top, free-slip side walls, a
    bubble of R = 0.25 m (nx/4 nodes) centred at (0.5 m, 0.5 m), gravity
    along -y; rho1/rho2 = 10 and mu1/mu2 = 10 (Table test_Paras, so equal
    kinematic viscosities), Re = rho1 Ug L / mu1 = 35, Eo = rho1 Ug^2 L /
    sigma = 10 with L = 2R and Ug = sqrt(2 R g).  Ug is the reference
    velocity in lattice units; the paper gives no mobility, interface width
    or tau_h.  The defaults are the ones every force form runs to t = 3 s
    with at 120 x 240: with W = 4, 5 or 6 phi undershoots -1 inside the
    light bubble until its density reaches zero and the run diverges
    (STF-1 at W = 4 after ~2400 steps, in the FP64 oracle as on the GPU).
    meta carries the lattice-to-SI conversions: seconds per step, metres
    per node, (m/s) per lattice velocity."""
    R = nx / 4.0
    L = 2.0 * R
    nu = Ug * L / Re
    sigma = Ug * Ug * L / Eo  # rho1 = 1
    g = Ug * Ug / (2.0 * R)
    p = dict(sigma=sigma, W=W, M=M, tau_h=tau_h, rho1=1.0, rho2=1.0 / rho_ratio,
             nu1=nu, nu2=nu * rho_ratio / mu_ratio, gx=0.0, gy=-g, form=form)
    ny = 2 * nx
    c = 0.5 * nx - 0.5  # node coordinate of 0.5 m
    dx, dy = _dist(nx, ny, c, c, False, False)
    phi0 = -np.tanh(2.0 * (R - np.sqrt(dx * dx + dy * dy)) / W)
    dx_m = 1.0 / nx
    return Case("rising_bubble", nx, ny, True, p, phi0, 0,
                {"R": R, "wall_x": True, "m_per_node": dx_m,
                 "s_per_step": dx_m * Ug / UG_PHYS, "mps_per_lattice": UG_PHYS / Ug})


def batch_instances(n=256, seed=0, sizes=(64, 128, 256, 512)):
    """Batched workload: n drop instances, L drawn from `sizes`, R uniform in
    [0.15, 0.35] L, sigma log-uniform in [1e-4, 1e-2], force family cycling
    STF, CPF, PF, CSF; odd instances are slightly elliptic (oscillating)."""
    rng = np.random.default_rng(seed)
    fams = ("STF1", "CPF1", "PF1", "CSF1")
    out = []
    for k in range(n):
        L = int(rng.choice(sizes))
        R = float(rng.uniform(0.15, 0.35) * L)
        sigma = float(10 ** rng.uniform(-4, -2))
        form = fams[k % 4]
        phi0 = ellipse(L, L, R, 4.0, 0.1) if k % 2 else drop(L, L, R, 4.0)
        p = dict(sigma=sigma, W=4.0, M=0.1, tau_h=1.0, rho1=1.0, rho2=1.0,
                 nu1=0.1, nu2=0.1, form=form)
        out.append(Case(f"inst{k}", L, L, False, p, phi0, 2000, {"R": R}))
    return out


def capillary_wave(form="STF1", H=80, h0_frac=0.02, Uc=0.01, rho_ratio=1.0, Re=50.0, We=1.0,
                   M=0.05, W=4.0):
    """H x 3H, walls at bottom and top, periodic sides; heavy fluid 1 below
    the interface y = 1.5 H + h0 cos(k x), k = 2 pi / H, h0 = h0_frac H
    (Sec. 5.3).  Parameters from the paper's groups Re = 50, We = 1 with
    Lc = H and a lattice reference velocity Uc (sigma = H Uc^2 / We, nu =
    Uc H / Re: 0.008 and 0.016 by default); equal kinematic viscosities (the
    analytic solution assumes them).  The mobility is set directly: the
    paper's default Pe = 1/Cn gives M = W We / (3 Uc Pe) = 6.7 here, for
    which the scheme diverges; M = 0.05 is Pe = 2667.  With Uc = 0.02 or
    0.05 (sigma = 0.032, 0.2) CPF-1 and PF-2 diverge, in the FP64 oracle as
    on the GPU."""
    from . import units
    Pe = W * We / (3.0 * Uc * M)
    p = units.lattice_params(Lc=H, Uc=Uc, Re=Re, We=We, Cn=W / H, Pe=Pe, rho_ratio=rho_ratio,
                             mu_ratio=rho_ratio)
    p["form"] = form
    nx, ny = H, 3 * H
    x, y = _grid(nx, ny)
    h0 = h0_frac * H
    # walls at y = -1/2 and ny - 1/2: height Y = y + 1/2 above the bottom wall
    yi = 1.5 * H - 0.5 + h0 * np.cos(2.0 * math.pi * x / nx)
    phi0 = np.tanh(2.0 * (yi - y) / W)
    return Case("capillary_wave", nx, ny, True, p, phi0, 0,
                {"h0": h0, "k": 2.0 * math.pi / H, "Uc": Uc})


def shear_drop(form="STF1", nx=512, ny=256, R=40.0, U=0.01, W=4.0, M=0.05,
               Re=1.0, Ca=0.2):
    """512x256, walls moving at +U (top) and -U (bottom), drop R = 40 at the
    centre, rho1 = rho2 = 1; nu from Re = E R^2/nu and sigma from
    Ca = nu E R / sigma with E = 2U/ny (Sec. 5.5)."""
    E = 2 * U / ny
    nu = E * R * R / Re
    sigma = nu * E * R / Ca
    p = dict(sigma=sigma, W=W, M=M, tau_h=1.0, rho1=1.0, rho2=1.0, nu1=nu, nu2=nu,
             uw_bottom=-U, uw_top=U, form=form)
    return Case("shear_drop", nx, ny, True, p, drop(nx, ny, R, W, periodic_y=False),
                4000, {"R": R, "E": E})

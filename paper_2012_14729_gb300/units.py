"""Dimensionless front-end: the paper's dimensionless groups (Sec. 2.3) to
lattice parameters for `pflbm.Domain.set_params`.

With the reference density and dynamic viscosity of fluid 1 (rho_c = rho1,
mu_c = mu1 = rho1 nu1), a reference length Lc (lattice nodes) and velocity
Uc (lattice units), the groups are

    Re = rho1 Uc Lc / mu1        Pe = Uc Lc / (4 M beta)     We = rho1 Lc Uc^2 / sigma
    Fr = Uc / sqrt(g Lc)         Cn = W / Lc

with beta = 3 sigma / (4 W) the free-energy coefficient (Sec. 2.1).  The
rising bubble (Sec. 5.4) is stated with Re and the Eotvos and Morton numbers

    Eo = rho1 g Lc^2 / sigma     Mo = Eo^3 / Re^4 = g mu1^4 / (rho1 sigma^3)

which are We and Re with the gravity velocity Uc = sqrt(g Lc) (Fr = 1).
"""
from __future__ import annotations

import math
from typing import Optional


def lattice_params(Lc: float, Uc: float, Re: float, We: float, Cn: float,
                   Pe: Optional[float] = None, Fr: Optional[float] = None,
                   rho1: float = 1.0, rho_ratio: float = 1.0, mu_ratio: float = 1.0,
                   tau_h: float = 1.0) -> dict:
    """Lattice parameters from the groups.  rho_ratio = rho1 / rho2 and
    mu_ratio = mu1 / mu2; Pe defaults to 1 / Cn (the paper's default, Sec. 5);
    Fr = None means no gravity (g acts along -y otherwise)."""
    if min(Lc, Uc, Re, We, Cn, rho1, rho_ratio, mu_ratio) <= 0:
        raise ValueError("Lc, Uc, Re, We, Cn and the ratios must be positive")
    Pe = 1.0 / Cn if Pe is None else Pe
    W = Cn * Lc
    sigma = rho1 * Lc * Uc * Uc / We
    nu1 = Uc * Lc / Re
    rho2 = rho1 / rho_ratio
    nu2 = (rho1 * nu1 / mu_ratio) / rho2
    beta = 3.0 * sigma / (4.0 * W)
    M = Uc * Lc / (4.0 * beta * Pe)
    gy = 0.0 if Fr is None else -Uc * Uc / (Fr * Fr * Lc)
    return dict(sigma=sigma, W=W, M=M, tau_h=tau_h, rho1=rho1, rho2=rho2, nu1=nu1, nu2=nu2,
                gx=0.0, gy=gy)


def groups(p: dict, Lc: float, Uc: float) -> dict:
    """The dimensionless groups of a parameter set (inverse of lattice_params)."""
    beta = 3.0 * p["sigma"] / (4.0 * p["W"])
    mu1 = p["rho1"] * p["nu1"]
    g = math.hypot(p.get("gx", 0.0), p.get("gy", 0.0))
    Eo = p["rho1"] * g * Lc * Lc / p["sigma"]
    return dict(Re=p["rho1"] * Uc * Lc / mu1, Pe=Uc * Lc / (4.0 * p["M"] * beta),
                We=p["rho1"] * Lc * Uc * Uc / p["sigma"],
                Fr=(Uc / math.sqrt(g * Lc)) if g > 0 else math.inf, Cn=p["W"] / Lc,
                rho_ratio=p["rho1"] / p["rho2"], mu_ratio=mu1 / (p["rho2"] * p["nu2"]),
                Eo=Eo, Mo=g * mu1 ** 4 / (p["rho1"] * p["sigma"] ** 3))

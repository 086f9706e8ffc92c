"""FP64 CPU oracle of the phase-field LBM coupled step (arXiv 2012.14729, Sec. 3).

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, plain reference the CUDA
path is checked against; only the tests, the smoke check and the benchmark's
CPU-baseline leg may import it.  It shares no code with the CUDA library.

The arithmetic lives in ``pflbm_oracle.c`` (plain loops, double precision,
whole-grid passes in the order of the scheme); this module compiles it with
gcc, calls it through ctypes, and adds the FP64 diagnostics of Sec. 5
(Laplace pressure jump, spurious currents, mass, mass centre, Taylor
deformation, the rising-bubble centre of mass, velocity and circularity with
a marching-squares perimeter), written with numpy and plain loops.

Parity of every function here is pinned by ``tests/test_oracle_*.py``
against moment identities, closed forms, invariants and physical laws.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pflbm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

FORMS = ("STF1", "STF2", "CPF1", "CPF2", "PF1", "PF2", "CSF1", "CSF2")
FAMILY = {"STF": "STF1", "CPF": "CPF1", "PF": "PF1", "CSF": "CSF1"}

# parameter vector layout shared with pflbm_oracle.c (P_* enum there)
_PAR = ("sigma", "W", "M", "tau_h", "rho1", "rho2", "nu1", "nu2", "gx", "gy",
        "rho0", "uw_bottom", "uw_top", "eps", "form")
# macro field block layout (M_* enum in pflbm_oracle.c)
FIELDS = ("phi", "gx", "gy", "lap", "mu", "Fx", "Fy", "rho", "ux", "uy", "P",
          "phiux", "phiuy", "div_phiu", "dt_phiux", "dt_phiuy", "tau_f", "p_h")

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


_SRC32 = os.path.join(_HERE, "pflbm_oracle_f32.c")
_LIB32 = os.path.join(_BUILD, "liboracle_f32.so")


def _compile(src: str, lib: str, force: bool) -> str:
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(src))
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= newest:
        return lib
    os.makedirs(_BUILD, exist_ok=True)
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-std=c99", "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -O2, OpenMP,
    no FMA contraction so results do not depend on the host ISA), and its
    float32-state build ``liboracle_f32.so``."""
    _compile(_SRC32, _LIB32, force)
    return _compile(_SRC, _LIB, force)


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        i = ctypes.c_int
        d = ctypes.c_double
        _lib.orc_feq.argtypes = [d, d, d, d, dp]
        _lib.orc_heq.argtypes = [d, d, d, d, d, dp]
        _lib.orc_fforce.argtypes = [d, d, d, d, d, d, dp]
        _lib.orc_hsource.argtypes = [d, d, d, d, dp]
        _lib.orc_macro.argtypes = [dp, i, i, i, dp, dp, dp, i, dp]
        _lib.orc_step.argtypes = [dp, i, i, i, dp, dp, dp, i, i]
        _lib.orc_init.argtypes = [dp, i, i, i, dp, dp, dp, dp]
        _lib.orc_ics.argtypes = [i, i, i, dp, dp]
        assert _lib.orc_nfields() == len(FIELDS)
        assert _lib.orc_npar() == len(_PAR)
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def set_threads(n: int) -> None:
    """Threads the oracle's OpenMP loops use (results do not depend on it)."""
    os.environ["OMP_NUM_THREADS"] = str(n)
    try:
        ctypes.CDLL("libgomp.so.1").omp_set_num_threads(int(n))
    except OSError:
        pass


@dataclass
class Params:
    """Physical parameters in lattice units (delta x = delta t = 1).

    sigma, W        surface tension and interface width (beta = 3 sigma / 4W,
                    kappa = 3 W sigma / 8, Sec. 2.1)
    M, tau_h        mobility and CH relaxation time (M = cs^2 eta (tau_h - 1/2))
    rho1, rho2      densities of fluid 1 (phi = +1) and fluid 2 (phi = -1)
    nu1, nu2        kinematic viscosities (mu_k = rho_k nu_k)
    gx, gy          gravity; F_g = (rho - rho0) g
    rho0            background density; NaN means the mean of rho(phi0)
    uw_bottom/top   x-velocity of the walls at y = -1/2 and y = ny - 1/2
    eps             regularisation of the CSF normal
    form            interfacial force formulation, one of FORMS
    """
    sigma: float = 0.01
    W: float = 4.0
    M: float = 0.1
    tau_h: float = 1.0
    rho1: float = 1.0
    rho2: float = 1.0
    nu1: float = 0.1
    nu2: float = 0.1
    gx: float = 0.0
    gy: float = 0.0
    rho0: float = float("nan")
    uw_bottom: float = 0.0
    uw_top: float = 0.0
    eps: float = 1e-6
    form: str = "STF1"

    def vector(self) -> np.ndarray:
        v = []
        for k in _PAR:
            val = getattr(self, k)
            if k == "form":
                val = FORMS.index(FAMILY.get(val, val))
            v.append(float(val))
        return np.array(v, dtype=np.float64)


def feq(P, rho, ux, uy):
    out = np.zeros(9)
    lib().orc_feq(P, rho, ux, uy, _p(out))
    return out


def heq(phi, mu, eta, ux, uy):
    out = np.zeros(9)
    lib().orc_heq(phi, mu, eta, ux, uy, _p(out))
    return out


def fforce(ux, uy, Fx, Fy, drx, dry):
    out = np.zeros(9)
    lib().orc_fforce(ux, uy, Fx, Fy, drx, dry, _p(out))
    return out


def hsource(tau_h, divphiu, dtx, dty):
    out = np.zeros(9)
    lib().orc_hsource(tau_h, divphiu, dtx, dty, _p(out))
    return out


def ics(a: np.ndarray, wall: bool = False):
    """Central-scheme gradient and Laplacian of a [ny][nx] field."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    ny, nx = a.shape
    out = np.zeros((3, ny, nx))
    lib().orc_ics(nx, ny, int(wall), _p(a), _p(out))
    return out[0], out[1], out[2]


def mean_rho(par: Params, phi0: np.ndarray) -> float:
    """Default background density: the domain mean of rho(phi0)."""
    rho = par.rho1 * 0.5 * (1 + phi0) + par.rho2 * 0.5 * (1 - phi0)
    return float(np.mean(rho))


class Sim:
    """One oracle run: pre-collision populations f, h at the current time,
    (phi u) of the previous step, and the step counter."""

    def __init__(self, nx: int, ny: int, wall_y: bool, par: Params, phi0: np.ndarray,
                 wall_x: bool = False):
        # boundary flags of the C oracle: bit 0 no-slip walls in y, bit 1
        # free-slip (mirror-symmetry) walls in x
        self.nx, self.ny = int(nx), int(ny)
        self.wall = (1 if wall_y else 0) | (2 if wall_x else 0)
        if wall_x and (par.gx != 0.0 or par.uw_bottom != 0.0 or par.uw_top != 0.0):
            # x-odd forcing would break the mirror symmetry that defines the walls
            raise ValueError("free-slip side walls need gx = 0 and walls at rest in y")
        phi0 = np.ascontiguousarray(phi0, dtype=np.float64).reshape(ny, nx)
        if math.isnan(par.rho0):
            par = Params(**{**par.__dict__, "rho0": mean_rho(par, phi0)})
        self.par = par
        self.pv = par.vector()
        self.f = np.zeros((9, ny, nx))
        self.h = np.zeros((9, ny, nx))
        self.phiu_prev = np.zeros((2, ny, nx))
        lib().orc_init(_p(self.pv), nx, ny, int(self.wall), _p(phi0), _p(self.f),
                       _p(self.h), _p(self.phiu_prev))
        self.t = 0

    def step(self, n: int = 1) -> "Sim":
        if n > 0:
            lib().orc_step(_p(self.pv), self.nx, self.ny, int(self.wall), _p(self.f),
                           _p(self.h), _p(self.phiu_prev), int(n), int(self.t == 0))
            self.t += n
        return self

    def macro(self) -> dict:
        out = np.zeros((len(FIELDS), self.ny, self.nx))
        lib().orc_macro(_p(self.pv), self.nx, self.ny, int(self.wall), _p(self.f),
                        _p(self.h), _p(self.phiu_prev), int(self.t == 0), _p(out))
        return {k: out[i] for i, k in enumerate(FIELDS)}


# ---------------------------------------------------------------------------
# FP64 diagnostics (Sec. 5)
# ---------------------------------------------------------------------------

def laplace(fields: dict, xc: float, yc: float, R: float, W: float,
            wrap_x: bool = True, wrap_y: bool = True) -> dict:
    """Laplace-law measurement (Sec. 5.1): R_num from the drop area, Delta p as
    the mean hydrodynamic pressure p_h inside r <= R/2 minus its mean outside
    r >= R + 3W (distance from the initial centre, periodic across the sides
    that are periodic), sigma_num = R_num Delta p."""
    phi, P = fields["phi"], fields["p_h"]
    ny, nx = phi.shape
    x = np.arange(nx)[None, :]
    y = np.arange(ny)[:, None]
    dx = np.abs(x - xc)
    if wrap_x:
        dx = np.minimum(dx, nx - dx)
    dy = np.abs(y - yc)
    if wrap_y:
        dy = np.minimum(dy, ny - dy)
    r = np.sqrt(dx * dx + dy * dy)
    inside = r <= R / 2
    outside = r >= R + 3 * W
    area = float(np.sum(0.5 * (1 + phi)))
    R_num = math.sqrt(area / math.pi)
    dp = float(P[inside].mean() - P[outside].mean())
    return {"R_num": R_num, "dp": dp, "sigma_num": R_num * dp}


def umax(fields: dict) -> float:
    return float(np.sqrt(fields["ux"] ** 2 + fields["uy"] ** 2).max())


def mass(fields: dict) -> float:
    return float(np.sum(fields["phi"]))


def mass_centre_x(fields: dict) -> float:
    """x_c of fluid 1 (weight (1 + phi)/2), Sec. 5.2."""
    w = 0.5 * (1 + fields["phi"])
    nx = w.shape[1]
    x = np.arange(nx)[None, :]
    return float(np.sum(w * x) / np.sum(w))


def taylor_D(fields: dict) -> float:
    """Taylor deformation D = (L - B)/(L + B) (Sec. 5.5), with L, B read as
    4 sqrt(lambda) of the second-moment matrix of w = (1 + phi)/2 about its
    centroid (twice the semi-axes of the equivalent ellipse)."""
    w = 0.5 * (1 + fields["phi"])
    ny, nx = w.shape
    x = np.arange(nx)[None, :] + 0.0 * w
    y = np.arange(ny)[:, None] + 0.0 * w
    m = w.sum()
    cx, cy = (w * x).sum() / m, (w * y).sum() / m
    sxx = (w * (x - cx) ** 2).sum() / m
    syy = (w * (y - cy) ** 2).sum() / m
    sxy = (w * (x - cx) * (y - cy)).sum() / m
    tr, det = sxx + syy, sxx * syy - sxy * sxy
    disc = math.sqrt(max(tr * tr / 4 - det, 0.0))
    l1, l2 = tr / 2 + disc, tr / 2 - disc
    L, B = 4 * math.sqrt(l1), 4 * math.sqrt(max(l2, 0.0))
    return (L - B) / (L + B)


def _crossing(p, vp, q, vq):
    """Point where the linear interpolant of phi between lattice points p and
    q (values vp, vq of opposite side of zero) vanishes."""
    t = vp / (vp - vq)
    return (p[0] + t * (q[0] - p[0]), p[1] + t * (q[1] - p[1]))


def _seg(a, b):
    return math.hypot(a[0] - b[0], a[1] - b[1])


def cell_contour_length(v) -> float:
    """Length of the phi = 0 contour inside one lattice cell by marching
    squares: v = (phi at (0,0), (1,0), (1,1), (0,1)), a corner is inside the
    bubble when phi < 0, the contour crosses each edge whose ends differ at
    the zero of the linear interpolant.  A cell with four crossings (inside
    corners on one diagonal) is resolved by the mean of its four values: if
    it is inside, the inside corners connect through the cell and each
    segment cuts off an outside corner; otherwise each cuts off an inside
    corner."""
    P = ((0.0, 0.0), (1.0, 0.0), (1.0, 1.0), (0.0, 1.0))
    ins = [x < 0 for x in v]
    pts = {}  # edge k joins corner k and corner k+1
    for k in range(4):
        j = (k + 1) % 4
        if ins[k] != ins[j]:
            pts[k] = _crossing(P[k], v[k], P[j], v[j])
    if len(pts) == 0:
        return 0.0
    if len(pts) == 2:
        a, b = pts.values()
        return _seg(a, b)
    centre_in = (v[0] + v[1] + v[2] + v[3]) / 4.0 < 0
    total = 0.0
    for k in range(4):
        if ins[k] != centre_in:  # the corner each segment cuts off
            total += _seg(pts[(k - 1) % 4], pts[k])
    return total


def contour_length(phi: np.ndarray, wrap_x: bool, wrap_y: bool) -> float:
    """Perimeter P_b of the bubble (Eq. circularity): the phi = 0 contour
    over the cells of the node lattice (spacing 1), a cell per node with the
    node as its lower-left corner; a periodic direction adds the cells that
    wrap around, a wall direction has none beyond the last node."""
    ny, nx = phi.shape
    cx = nx if wrap_x else nx - 1
    cy = ny if wrap_y else ny - 1
    total = 0.0
    for y in range(cy):
        y1 = (y + 1) % ny
        for x in range(cx):
            x1 = (x + 1) % nx
            v = (phi[y, x], phi[y, x1], phi[y1, x1], phi[y1, x])
            if min(v) < 0 <= max(v):
                total += cell_contour_length(v)
    return total


def rising_bubble(fields: dict, wall_x: bool, wall_y: bool) -> dict:
    """Benchmark quantities of the rising bubble (Sec. 5.4), lattice units:
    centre of mass (xc2, yc2) and velocity (uc2, vc2) of fluid 2 weighted by
    1 - phi (Eqs. quantify-yc, quantify-uc, node coordinates x, y), the area
    area2 = number of nodes with phi < 0, the perimeter of the phi = 0
    contour and the circularity 2 sqrt(pi area2) / perimeter (Eq.
    circularity; 0 when there is no contour; the means are 0 when no node
    holds fluid 2)."""
    phi = fields["phi"]
    ny, nx = phi.shape
    w = 1.0 - phi
    x = np.arange(nx)[None, :] + 0.0 * w
    y = np.arange(ny)[:, None] + 0.0 * w
    m = w.sum()
    area2 = float(np.count_nonzero(phi < 0))
    per = contour_length(phi, not wall_x, not wall_y)

    def mean(q):
        return float((w * q).sum() / m) if m > 0 else 0.0
    return {"mass2": float(m), "xc2": mean(x), "yc2": mean(y),
            "uc2": mean(fields["ux"]), "vc2": mean(fields["uy"]),
            "area2": area2, "perimeter": per,
            "circularity": 2.0 * math.sqrt(math.pi * area2) / per if per > 0 else 0.0}


# ---------------------------------------------------------------------------
# float32 rounding sensitivity of a workload
# ---------------------------------------------------------------------------

_lib32 = None


def lib32():
    global _lib32
    if _lib32 is None:
        build()
        _lib32 = ctypes.CDLL(_LIB32)
        dp = ctypes.POINTER(ctypes.c_double)
        i = ctypes.c_int
        _lib32.w32_step.argtypes = [dp, i, i, i, dp, dp, dp, i, i]
        _lib32.w32_macro.argtypes = [dp, i, i, i, dp, dp, dp, i, dp]
    return _lib32


def float32_deviation(nx, ny, wall_y, par: Params, phi0, steps: int, wall_x: bool = False) -> dict:
    """Max |phi| and |u| deviation after `steps` steps between the FP64 oracle
    and the same algorithm run with float32 state (pflbm_oracle_f32.c), both
    from phi0.  It measures the rounding sensitivity of a workload, from which
    tests derive the tolerance of a float32 implementation."""
    a = Sim(nx, ny, wall_y, par, phi0, wall_x)
    b = Sim(nx, ny, wall_y, par, phi0, wall_x)
    a.step(steps)
    L = lib32()
    L.w32_step(_p(b.pv), b.nx, b.ny, int(b.wall), _p(b.f), _p(b.h), _p(b.phiu_prev),
               int(steps), 1)
    out = np.zeros((len(FIELDS), ny, nx))
    L.w32_macro(_p(b.pv), b.nx, b.ny, int(b.wall), _p(b.f), _p(b.h), _p(b.phiu_prev),
                int(steps == 0), _p(out))
    m = a.macro()
    f32 = {k: out[i] for i, k in enumerate(FIELDS)}
    return {
        "phi": float(np.abs(f32["phi"] - m["phi"]).max()),
        "u": float(max(np.abs(f32["ux"] - m["ux"]).max(), np.abs(f32["uy"] - m["uy"]).max())),
        "fields64": m,
    }

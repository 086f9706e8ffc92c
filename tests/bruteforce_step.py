"""A second, independent transcription of one time step of the phase-field
lattice Boltzmann method (Zhang, Liang & Guo, arXiv 2012.14729, Sec. 3 and
Sec. 4), in plain Python: nested lists, scalar loops, no numpy in the
arithmetic and nothing imported from the oracle.  Tests compare it with the
oracle on lattices of a few nodes, where it runs in well under a second.

It is organised differently from the oracle on purpose:
  - every scalar field is a function of a node of the *extended* lattice;
    a node beyond a wall or a periodic seam is mapped back into the domain
    (mirror ghosts about the wall planes, Sec. 4; wrap for periodic sides)
    and the derived fields (grad phi, lap phi, mu, the force-form fields)
    are evaluated there by applying the stencils to the mapped phi, instead
    of mirroring stored derived fields with a parity sign;
  - grad rho is the central-scheme gradient of the rho field itself (rho is
    linear in phi, so this equals the chain rule up to rounding);
  - the collision is written as the paper prints it, f_i - (f_i - f_i^eq) /
    tau_f + (1 - 1/(2 tau_f)) F_i with F_i = (c_i - u) . [Gamma_i F +
    w_i s_i grad(cs^2 rho)], Gamma_i = w_i (1 + s_i) (the reading of Eq.
    P_LBM whose moments match Eq. mac);
  - streaming is a push of each post-collision population, with Ladd's
    half-way bounce-back at the y walls (Sec. 4) and specular reflection at
    free-slip side walls (Sec. 5.4).

Readings it shares with the oracle (they are the paper's gaps, stated once
for both): mirror ghosts with y-odd quantities negated, the ghost of phi u
next to a wall is phi (2 u_w - u) of the mirrored node, d_t(phi u) is the
one-step backward difference (zero at the first step), the CSF normal is
grad phi / sqrt(|grad phi|^2 + eps^2).
"""
import math

CS2 = 1.0 / 3.0
C = ((0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1))
W = (4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
     1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0)


def opposite(i):
    cx, cy = C[i]
    return C.index((-cx, -cy))


def x_mirror(i):
    cx, cy = C[i]
    return C.index((-cx, cy))


class Lattice:
    """nx x ny nodes; wall_y: no-slip walls at y = -1/2 and ny - 1/2 (else
    periodic in y); wall_x: free-slip walls at x = -1/2 and nx - 1/2 (else
    periodic in x)."""

    def __init__(self, nx, ny, wall_y, wall_x=False):
        self.nx, self.ny, self.wall_y, self.wall_x = nx, ny, wall_y, wall_x

    @staticmethod
    def _fold(v, n, mirror):
        """Index in [0, n) of extended index v, and how many mirror images
        were crossed (odd: the image is reflected)."""
        if not mirror:
            return v % n, 0
        flips = 0
        while v < 0 or v >= n:
            v = -1 - v if v < 0 else 2 * n - 1 - v
            flips += 1
        return v, flips

    def node(self, x, y):
        """(x, y) folded into the domain, with the parity of the x and y
        reflections (1 or -1)."""
        xx, fx = self._fold(x, self.nx, self.wall_x)
        yy, fy = self._fold(y, self.ny, self.wall_y)
        return xx, yy, (-1) ** fx, (-1) ** fy


def ics_grad(fn, x, y):
    """Eq. ICS-1st: grad Psi = (1/cs^2) sum_{i=1..8} w_i c_i Psi(x + c_i)."""
    sx = sy = 0.0
    for i in range(1, 9):
        cx, cy = C[i]
        v = fn(x + cx, y + cy)
        sx += W[i] * cx * v
        sy += W[i] * cy * v
    return sx / CS2, sy / CS2


def ics_lap(fn, x, y):
    """Eq. ICS-sec: lap Psi = (2/cs^2) sum_{i=1..8} w_i [Psi(x + c_i) - Psi(x)]."""
    c = fn(x, y)
    s = 0.0
    for i in range(1, 9):
        cx, cy = C[i]
        s += W[i] * (fn(x + cx, y + cy) - c)
    return 2.0 * s / CS2


def ics_div(fx, fy, x, y):
    """Divergence by Eq. ICS-1st applied to each component."""
    s = 0.0
    for i in range(1, 9):
        cx, cy = C[i]
        s += W[i] * (cx * fx(x + cx, y + cy) + cy * fy(x + cx, y + cy))
    return s / CS2


def step(lat, par, f, h, phiu_prev, first):
    """One time step.  f, h: [9][ny][nx] pre-collision populations at t (nested
    lists); phiu_prev: [2][ny][nx] (phi u)^{t-1}; par: dict with sigma, W, M,
    tau_h, rho1, rho2, nu1, nu2, gx, gy, rho0, uw_bottom, uw_top, eps, form.
    Returns (f, h, phiu) at t + 1 (phiu = (phi u)^t)."""
    nx, ny = lat.nx, lat.ny
    sigma, Wd = par["sigma"], par["W"]
    beta = 3.0 * sigma / (4.0 * Wd)          # Sec. 2.1
    kappa = 3.0 * Wd * sigma / 8.0
    rho1, rho2 = par["rho1"], par["rho2"]
    tau_h = par["tau_h"]
    eta = par["M"] / (CS2 * (tau_h - 0.5))   # M = cs^2 eta (tau_h - 1/2)
    form = par["form"]
    eps = par["eps"]

    memo = {}

    def cached(name, fn):
        def g(x, y):
            key = (name, x, y)
            if key not in memo:
                memo[key] = fn(x, y)
            return memo[key]
        return g

    # phi = sum_i h_i (Eq. mac) at a domain node; even under every mirror
    def phi_dom(x, y):
        return sum(h[i][y][x] for i in range(9))

    def phi(x, y):
        xx, yy, _, _ = lat.node(x, y)
        return phi_dom(xx, yy)
    phi = cached("phi", phi)

    def rho_of(p):
        return rho1 * (1.0 + p) / 2.0 + rho2 * (1.0 - p) / 2.0

    def rho(x, y):
        return rho_of(phi(x, y))

    grad_phi = cached("gphi", lambda x, y: ics_grad(phi, x, y))
    lap_phi = cached("lphi", lambda x, y: ics_lap(phi, x, y))

    # Eq. chemical_potential with f0 = beta (1 - phi^2)^2
    def mu(x, y):
        p = phi(x, y)
        return -4.0 * beta * p * (1.0 - p * p) - kappa * lap_phi(x, y)
    mu = cached("mu", mu)

    def gx(x, y):
        return grad_phi(x, y)[0]

    def gy(x, y):
        return grad_phi(x, y)[1]

    def normal(x, y):
        a, b = grad_phi(x, y)
        d = math.sqrt(a * a + b * b + eps * eps)
        return a / d, b / d
    normal = cached("n", normal)

    def interfacial(x, y):
        """F_sf of the selected formulation (Sec. 2.2), each written as its
        equation with the central scheme for every derivative."""
        a, b = grad_phi(x, y)
        if form in ("STF1", "STF2"):
            # -kappa div(grad phi (x) grad phi): component a = d_b (g_a g_b)
            Fx = -kappa * ics_div(lambda u, v: gx(u, v) * gx(u, v),
                                  lambda u, v: gx(u, v) * gy(u, v), x, y)
            Fy = -kappa * ics_div(lambda u, v: gy(u, v) * gx(u, v),
                                  lambda u, v: gy(u, v) * gy(u, v), x, y)
            if form == "STF2":
                # + kappa div(|grad phi|^2 I) = kappa grad |grad phi|^2
                sx, sy = ics_grad(lambda u, v: gx(u, v) ** 2 + gy(u, v) ** 2, x, y)
                Fx += kappa * sx
                Fy += kappa * sy
            return Fx, Fy
        if form == "CPF1":
            mx, my = ics_grad(mu, x, y)
            return -phi(x, y) * mx, -phi(x, y) * my
        if form == "CPF2":
            return mu(x, y) * a, mu(x, y) * b
        if form == "PF1":
            return -kappa * a * lap_phi(x, y), -kappa * b * lap_phi(x, y)
        if form == "PF2":
            lx, ly = ics_grad(lap_phi, x, y)
            return kappa * phi(x, y) * lx, kappa * phi(x, y) * ly
        divn = ics_div(lambda u, v: normal(u, v)[0], lambda u, v: normal(u, v)[1], x, y)
        if form == "CSF1":
            g = math.sqrt(a * a + b * b)
            return -kappa * a * g * divn, -kappa * b * g * divn
        if form == "CSF2":
            return -0.5 * sigma * a * divn, -0.5 * sigma * b * divn
        raise ValueError(form)

    def force(x, y):
        """F = F_sf + F_g at a domain node, F_g = (rho - rho0) g (Eq. NS)."""
        Fx, Fy = interfacial(x, y)
        r = rho(x, y)
        return Fx + (r - par["rho0"]) * par["gx"], Fy + (r - par["rho0"]) * par["gy"]

    grad_rho = cached("grho", lambda x, y: ics_grad(rho, x, y))

    def velocity(x, y):
        """u = [sum c_i f_i + cs^2 F / 2] / (cs^2 rho) at a domain node (Eq. mac)."""
        jx = sum(C[i][0] * f[i][y][x] for i in range(9))
        jy = sum(C[i][1] * f[i][y][x] for i in range(9))
        Fx, Fy = force(x, y)
        r = rho(x, y)
        return (jx + 0.5 * CS2 * Fx) / (CS2 * r), (jy + 0.5 * CS2 * Fy) / (CS2 * r)
    velocity = cached("u", velocity)

    def phiu(x, y):
        """phi u at any node of the extended lattice: beyond a no-slip wall
        phi (2 u_w - u) of the mirrored node, beyond a free-slip side wall the
        mirror image (x component reversed)."""
        xx, yy, sx, _ = lat.node(x, 0 if lat.wall_y else y)
        if lat.wall_y and (y < 0 or y >= ny):
            uw = par["uw_bottom"] if y < 0 else par["uw_top"]
            ym = 0 if y < 0 else ny - 1
            # the mirrored node of a first ghost row is the first fluid row
            assert y in (-1, ny)
            ux, uy = velocity(xx, ym)
            p = phi(xx, ym)
            vx, vy = p * (2.0 * uw - ux), p * (0.0 - uy)
        else:
            xx, yy, sx, _ = lat.node(x, y)
            ux, uy = velocity(xx, yy)
            p = phi(xx, yy)
            vx, vy = p * ux, p * uy
        return sx * vx, vy

    fo = [[[0.0] * nx for _ in range(ny)] for _ in range(9)]
    ho = [[[0.0] * nx for _ in range(ny)] for _ in range(9)]
    out_phiu = [[[0.0] * nx for _ in range(ny)] for _ in range(2)]
    post_f = [[[0.0] * nx for _ in range(ny)] for _ in range(9)]
    post_h = [[[0.0] * nx for _ in range(ny)] for _ in range(9)]

    tau1 = tau_h - 0.5
    tau2 = tau_h * tau_h - tau_h + 1.0 / 6.0
    for y in range(ny):
        for x in range(nx):
            p = phi(x, y)
            r = rho(x, y)
            ux, uy = velocity(x, y)
            Fx, Fy = force(x, y)
            rx, ry = grad_rho(x, y)
            # Eq. mac: P = sum f + cs^2/2 u . grad rho
            P = sum(f[i][y][x] for i in range(9)) + 0.5 * CS2 * (ux * rx + uy * ry)
            mv = rho1 * par["nu1"] * (1.0 + p) / 2.0 + rho2 * par["nu2"] * (1.0 - p) / 2.0
            tau_f = 0.5 + mv / (r * CS2)      # mu = rho cs^2 (tau_f - 1/2)
            pux, puy = p * ux, p * uy
            out_phiu[0][y][x], out_phiu[1][y][x] = pux, puy
            div = ics_div(lambda u, v: phiu(u, v)[0], lambda u, v: phiu(u, v)[1], x, y)
            if first:
                dtx = dty = 0.0
            else:
                dtx, dty = pux - phiu_prev[0][y][x], puy - phiu_prev[1][y][x]
            m = mu(x, y)
            uu = ux * ux + uy * uy
            for i in range(9):
                cx, cy = C[i]
                cu = cx * ux + cy * uy
                # s_i = c.u/cs^2 + uu:(cc - cs^2 I)/(2 cs^4)
                s = cu / CS2 + ((cx * cx - CS2) * ux * ux + 2 * cx * cy * ux * uy +
                                (cy * cy - CS2) * uy * uy) / (2.0 * CS2 * CS2)
                feq = W[i] * (P + CS2 * r * s)
                gam = W[i] * (1.0 + s)
                Fi = (cx - ux) * (gam * Fx + W[i] * s * CS2 * rx) + \
                     (cy - uy) * (gam * Fy + W[i] * s * CS2 * ry)
                fi = f[i][y][x]
                post_f[i][y][x] = fi - (fi - feq) / tau_f + (1.0 - 1.0 / (2.0 * tau_f)) * Fi
                # Eq. heq_CH and Eq. CH_LB_force (wbar_0 = w_0 - 1, wbar_i = w_i)
                if i == 0:
                    heq = p + (W[0] - 1.0) * eta * m
                    wbar = W[0] - 1.0
                else:
                    heq = W[i] * eta * m + W[i] * p * cu / CS2
                    wbar = W[i]
                Hi = wbar * 3.0 * tau2 / (tau_h * tau1) * div + W[i] * (cx * dtx + cy * dty) / CS2
                hi = h[i][y][x]
                post_h[i][y][x] = hi - (hi - heq) / tau_h + (1.0 - 1.0 / (2.0 * tau_h)) * Hi

    # streaming: push; Ladd bounce-back at the y walls, specular reflection
    # at free-slip side walls
    for y in range(ny):
        for x in range(nx):
            for i in range(9):
                cx, cy = C[i]
                tx, ty = x + cx, y + cy
                if lat.wall_y and (ty < 0 or ty >= ny):
                    uw = par["uw_bottom"] if ty < 0 else par["uw_top"]
                    cuw = cx * uw
                    j = opposite(i)
                    fo[j][y][x] = post_f[i][y][x] - 2.0 * W[i] * rho(x, y) * cuw
                    ho[j][y][x] = post_h[i][y][x] - 2.0 * W[i] * phi(x, y) * cuw / CS2
                    continue
                if lat.wall_x and (tx < 0 or tx >= nx):
                    j = x_mirror(i)
                    fo[j][ty % ny][x] = post_f[i][y][x]
                    ho[j][ty % ny][x] = post_h[i][y][x]
                    continue
                fo[i][ty % ny][tx % nx] = post_f[i][y][x]
                ho[i][ty % ny][tx % nx] = post_h[i][y][x]
    return fo, ho, out_phiu


def run(lat, par, f, h, phiu_prev, first, nsteps):
    for s in range(nsteps):
        f, h, phiu_prev = step(lat, par, f, h, phiu_prev, first and s == 0)
    return f, h, phiu_prev

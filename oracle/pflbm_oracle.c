/*
 * FP64 CPU oracle of one coupled time step of the phase-field lattice
 * Boltzmann method of Zhang, Liang & Guo, "On the formulations of interfacial
 * force in the phase-field-based lattice Boltzmann method" (arXiv 2012.14729).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it; the product path never does.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Every quantity is double precision.  Each step is a sequence of whole-grid
 * passes in the order the paper's scheme needs them (Sec. 3):
 *   1. phi = sum_i h_i                                      (Eq. mac)
 *   2. grad phi, lap phi by the isotropic central scheme    (Eqs. ICS-1st, ICS-sec)
 *   3. mu = 4 beta phi (phi^2 - 1) - kappa lap phi          (Eq. chemical_potential)
 *   4. interfacial force in the selected formulation        (Eqs. SF1, SF2, SF3456, SF7, SF8)
 *      plus gravity F_g = (rho - rho0) g                    (Eq. NS)
 *   5. rho, grad rho, tau_f, u, P                           (Sec. 2.1, Eq. mac)
 *   6. phi u, div(phi u), d_t(phi u)                        (Eq. CH_LB_force)
 *   7. BGK collision of f and h with forcing                (Eq. fh, P_LBM, CH_LB_force)
 *   8. streaming, periodic wrap or Ladd half-way bounce-back (Sec. 4)
 *   9. (phi u)^{t-1} <- (phi u)^t
 *
 * Readings of points the paper leaves open (each is stated where used):
 *   - Force term: Gamma_i = w_i (1 + s_i) and the grad rho coefficient is
 *     w_i s_i, so that sum_i F_i = u . grad(cs^2 rho) and
 *     sum_i c_i F_i = cs^2 F match the macroscopic relations of Eq. mac.
 *   - Each force formulation is discretised literally with the central
 *     scheme applied to node fields (nested stencils), no identities used.
 *   - CSF normal n = grad phi / sqrt(|grad phi|^2 + eps^2).
 *   - Walls (y = -1/2 and y = ny - 1/2): scalar stencils see mirror ghosts,
 *     ghost row -k equals row k-1 with y-odd quantities negated; the ghost of
 *     phi u is phi (2 u_w - u) of the mirrored node.
 *   - d_t(phi u) is the backward difference over one step, zero at the first
 *     step of a run.
 *   - Free-slip side walls (rising-bubble benchmark, Sec. 5.4): planes of
 *     mirror symmetry at x = -1/2 and nx - 1/2 (see orc_step below).
 *
 * Layout: populations are [9][ny][nx] row-major (x fastest), fields [ny][nx].
 * Direction order c_0..c_8 = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),
 * (-1,-1),(1,-1) with weights 4/9, 1/9 x4, 1/36 x4 (Sec. 3, D2Q9).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define NQ 9

static const int ex[NQ] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int ey[NQ] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double wq[NQ] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                              1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                              1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int opp[NQ] = {0, 3, 4, 1, 2, 7, 8, 5, 6};

/* parameter vector layout (doubles) */
enum {
  P_SIGMA = 0, P_W, P_M, P_TAUH, P_RHO1, P_RHO2, P_NU1, P_NU2, P_GX, P_GY,
  P_RHO0, P_UWB, P_UWT, P_EPS, P_FORM, P_NPAR
};

enum { STF1 = 0, STF2, CPF1, CPF2, PF1, PF2, CSF1, CSF2 };

typedef struct {
  int nx, ny, wall;
} Grid;

/* --------------------------------------------------------------------- */
/* boundary rule for scalar stencils                                      */
/* --------------------------------------------------------------------- */

static int wrapx(const Grid* g, int x) {
  x %= g->nx;
  return x < 0 ? x + g->nx : x;
}

/* Value of a node field at (x, y), y possibly outside [0, ny).  Periodic:
 * wrap.  Wall: mirror about the wall plane, ghost row -k = row k-1, with the
 * sign `parity` (+1 for quantities even in y, -1 for y-odd ones). */
static double at(const Grid* g, const double* a, int x, int y, double parity) {
  x = wrapx(g, x);
  if (!g->wall) {
    y %= g->ny;
    if (y < 0) y += g->ny;
    return a[(size_t)y * g->nx + x];
  }
  double s = 1.0;
  while (y < 0 || y >= g->ny) {
    if (y < 0) y = -y - 1;
    else y = 2 * g->ny - 1 - y;
    s *= parity;
  }
  return s * a[(size_t)y * g->nx + x];
}

/* Isotropic central scheme, Eq. ICS-1st: grad Psi = (1/cs^2) sum_{i>0} w_i c_i Psi(x+c_i). */
static void ics_grad_node(const Grid* g, const double* a, double parity, int x,
                          int y, double* gx, double* gy) {
  double sx = 0.0, sy = 0.0;
  for (int i = 1; i < NQ; ++i) {
    double v = at(g, a, x + ex[i], y + ey[i], parity);
    sx += wq[i] * ex[i] * v;
    sy += wq[i] * ey[i] * v;
  }
  *gx = 3.0 * sx;
  *gy = 3.0 * sy;
}

/* Isotropic central scheme, Eq. ICS-sec: lap Psi = (2/cs^2) sum_{i>0} w_i [Psi(x+c_i) - Psi(x)]. */
static double ics_lap_node(const Grid* g, const double* a, int x, int y) {
  double c = a[(size_t)y * g->nx + x];
  double s = 0.0;
  for (int i = 1; i < NQ; ++i) s += wq[i] * (at(g, a, x + ex[i], y + ey[i], 1.0) - c);
  return 6.0 * s;
}

/* x-component of grad of a field that is even in y, plus the y-component of
 * grad of a field with the given parity: used for divergences. */
static double ics_ddx(const Grid* g, const double* a, double parity, int x, int y) {
  double s = 0.0;
  for (int i = 1; i < NQ; ++i) s += wq[i] * ex[i] * at(g, a, x + ex[i], y + ey[i], parity);
  return 3.0 * s;
}
static double ics_ddy(const Grid* g, const double* a, double parity, int x, int y) {
  double s = 0.0;
  for (int i = 1; i < NQ; ++i) s += wq[i] * ey[i] * at(g, a, x + ex[i], y + ey[i], parity);
  return 3.0 * s;
}

/* --------------------------------------------------------------------- */
/* local (per node) pieces, exported for the moment tests                 */
/* --------------------------------------------------------------------- */

/* s_i(u) = c_i.u/cs^2 + uu:(c_i c_i - cs^2 I)/(2 cs^4)  (Sec. 3) */
static double s_i(int i, double ux, double uy) {
  double cu = ex[i] * ux + ey[i] * uy;
  return 3.0 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy);
}

/* f_i^eq = w_i [P + cs^2 rho s_i(u)] */
void orc_feq(double P, double rho, double ux, double uy, double* out) {
  for (int i = 0; i < NQ; ++i) out[i] = wq[i] * (P + rho / 3.0 * s_i(i, ux, uy));
}

/* h_i^eq, Eq. heq_CH */
void orc_heq(double phi, double mu, double eta, double ux, double uy, double* out) {
  out[0] = phi + (wq[0] - 1.0) * eta * mu;
  for (int i = 1; i < NQ; ++i)
    out[i] = wq[i] * eta * mu + wq[i] * phi * 3.0 * (ex[i] * ux + ey[i] * uy);
}

/* F_i, Eq. P_LBM with Gamma_i = w_i (1 + s_i) and grad-rho weight w_i s_i. */
void orc_fforce(double ux, double uy, double Fx, double Fy, double drx, double dry,
                double* out) {
  for (int i = 0; i < NQ; ++i) {
    double si = s_i(i, ux, uy);
    double ax = wq[i] * (1.0 + si) * Fx + wq[i] * si * drx / 3.0;
    double ay = wq[i] * (1.0 + si) * Fy + wq[i] * si * dry / 3.0;
    out[i] = (ex[i] - ux) * ax + (ey[i] - uy) * ay;
  }
}

/* H_i, Eq. CH_LB_force with wbar_0 = w_0 - 1, wbar_i = w_i (Sec. 5). */
void orc_hsource(double tau_h, double divphiu, double dtx, double dty, double* out) {
  double t1 = tau_h - 0.5;
  double t2 = tau_h * tau_h - tau_h + 1.0 / 6.0;
  double A = 3.0 * t2 / (tau_h * t1) * divphiu;
  for (int i = 0; i < NQ; ++i) {
    double wb = (i == 0) ? wq[0] - 1.0 : wq[i];
    out[i] = wb * A + wq[i] * 3.0 * (ex[i] * dtx + ey[i] * dty);
  }
}

/* --------------------------------------------------------------------- */
/* whole-grid macroscopic pass                                            */
/* --------------------------------------------------------------------- */

/* Field indices of the macro output block, each [ny][nx]. */
enum {
  M_PHI = 0, M_GX, M_GY, M_LAP, M_MU, M_FX, M_FY, M_RHO, M_UX, M_UY, M_P,
  M_PUX, M_PUY, M_DIV, M_DTX, M_DTY, M_TAUF, M_PH, M_NFIELDS
};

/* Form-specific level-1 fields. */
enum { X_TXX = 0, X_TXY, X_TYY, X_G2, X_NX, X_NY, X_NFIELDS };

static double beta_of(const double* p) { return 0.75 * p[P_SIGMA] / p[P_W]; }
static double kappa_of(const double* p) { return 0.375 * p[P_W] * p[P_SIGMA]; }

/* Interfacial force at one node, from level-1 fields (Sec. 2.2). */
static void force_sf(const Grid* g, const double* p, int form, const double* m,
                     const double* xf, int x, int y, double* Fx, double* Fy) {
  size_t n = (size_t)g->nx * g->ny;
  size_t k = (size_t)y * g->nx + x;
  const double* phi = m + M_PHI * n;
  const double* Gx = m + M_GX * n;
  const double* Gy = m + M_GY * n;
  const double* L = m + M_LAP * n;
  const double* mu = m + M_MU * n;
  double kap = kappa_of(p);
  double sig = p[P_SIGMA];
  switch (form) {
    case STF1:
    case STF2: {
      /* -div(kappa grad phi (x) grad phi): (div T)_a = d_x T_ax + d_y T_ay */
      const double* Txx = xf + X_TXX * n;
      const double* Txy = xf + X_TXY * n;
      const double* Tyy = xf + X_TYY * n;
      double dx = ics_ddx(g, Txx, 1.0, x, y) + ics_ddy(g, Txy, -1.0, x, y);
      double dy = ics_ddx(g, Txy, -1.0, x, y) + ics_ddy(g, Tyy, 1.0, x, y);
      *Fx = -kap * dx;
      *Fy = -kap * dy;
      if (form == STF2) {
        /* + div(kappa |grad phi|^2 I) = kappa grad |grad phi|^2 */
        const double* G2 = xf + X_G2 * n;
        *Fx += kap * ics_ddx(g, G2, 1.0, x, y);
        *Fy += kap * ics_ddy(g, G2, 1.0, x, y);
      }
      break;
    }
    case CPF1: { /* -phi grad mu */
      double gx, gy;
      ics_grad_node(g, mu, 1.0, x, y, &gx, &gy);
      *Fx = -phi[k] * gx;
      *Fy = -phi[k] * gy;
      break;
    }
    case CPF2: /* mu grad phi */
      *Fx = mu[k] * Gx[k];
      *Fy = mu[k] * Gy[k];
      break;
    case PF1: /* -kappa grad phi lap phi */
      *Fx = -kap * Gx[k] * L[k];
      *Fy = -kap * Gy[k] * L[k];
      break;
    case PF2: { /* kappa phi grad lap phi */
      double gx, gy;
      ics_grad_node(g, L, 1.0, x, y, &gx, &gy);
      *Fx = kap * phi[k] * gx;
      *Fy = kap * phi[k] * gy;
      break;
    }
    case CSF1:
    case CSF2: {
      const double* Nx = xf + X_NX * n;
      const double* Ny = xf + X_NY * n;
      double divn = ics_ddx(g, Nx, 1.0, x, y) + ics_ddy(g, Ny, -1.0, x, y);
      if (form == CSF1) {
        /* -kappa grad phi |grad phi| div n  (Dirac alpha |grad phi|^2, alpha = 3W/8) */
        double gabs = sqrt(Gx[k] * Gx[k] + Gy[k] * Gy[k]);
        *Fx = -kap * Gx[k] * gabs * divn;
        *Fy = -kap * Gy[k] * gabs * divn;
      } else {
        /* -(sigma/2) grad phi div n  (Dirac alpha |grad phi|, alpha = 1/2) */
        *Fx = -0.5 * sig * Gx[k] * divn;
        *Fy = -0.5 * sig * Gy[k] * divn;
      }
      break;
    }
    default:
      *Fx = 0.0;
      *Fy = 0.0;
  }
}

/* Macroscopic pass: every field of one time level from the pre-collision
 * populations f, h (post-streaming, time t) and (phi u)^{t-1}.
 * out: M_NFIELDS blocks of [ny][nx]. */
static void macro_px(const double* p, int nx, int ny, int wall, const double* f,
               const double* h, const double* phiu_prev, int first, double* out) {
  Grid g = {nx, ny, wall};
  size_t n = (size_t)nx * ny;
  int form = (int)p[P_FORM];
  double beta = beta_of(p), kap = kappa_of(p);
  double rho1 = p[P_RHO1], rho2 = p[P_RHO2];
  double* m = out;
  double* phi = m + M_PHI * n;
  double* xf = (double*)malloc(sizeof(double) * X_NFIELDS * n);

  /* 1. phi = sum_i h_i */
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t k = (size_t)y * nx + x;
      double s = 0.0;
      for (int i = 0; i < NQ; ++i) s += h[i * n + k];
      phi[k] = s;
    }

  /* 2-3. grad phi, lap phi, mu; level-1 fields of the force forms */
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t k = (size_t)y * nx + x;
      double gx, gy;
      ics_grad_node(&g, phi, 1.0, x, y, &gx, &gy);
      double L = ics_lap_node(&g, phi, x, y);
      double ph = phi[k];
      m[M_GX * n + k] = gx;
      m[M_GY * n + k] = gy;
      m[M_LAP * n + k] = L;
      m[M_MU * n + k] = 4.0 * beta * ph * (ph * ph - 1.0) - kap * L;
      xf[X_TXX * n + k] = gx * gx;
      xf[X_TXY * n + k] = gx * gy;
      xf[X_TYY * n + k] = gy * gy;
      xf[X_G2 * n + k] = gx * gx + gy * gy;
      double inv = 1.0 / sqrt(gx * gx + gy * gy + p[P_EPS] * p[P_EPS]);
      xf[X_NX * n + k] = gx * inv;
      xf[X_NY * n + k] = gy * inv;
    }

  /* 4-5. force, rho, u, P */
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t k = (size_t)y * nx + x;
      double Fx, Fy;
      force_sf(&g, p, form, m, xf, x, y, &Fx, &Fy);
      double ph = phi[k];
      double rho = rho1 * 0.5 * (1.0 + ph) + rho2 * 0.5 * (1.0 - ph);
      Fx += (rho - p[P_RHO0]) * p[P_GX];
      Fy += (rho - p[P_RHO0]) * p[P_GY];
      double mv = rho1 * p[P_NU1] * 0.5 * (1.0 + ph) + rho2 * p[P_NU2] * 0.5 * (1.0 - ph);
      double tauf = 0.5 + 3.0 * mv / rho;
      double sf = 0.0, jx = 0.0, jy = 0.0;
      for (int i = 0; i < NQ; ++i) {
        double v = f[i * n + k];
        sf += v;
        jx += ex[i] * v;
        jy += ey[i] * v;
      }
      /* u = [sum c f + cs^2 F / 2] / (cs^2 rho) */
      double ux = (jx + Fx / 6.0) / (rho / 3.0);
      double uy = (jy + Fy / 6.0) / (rho / 3.0);
      /* grad rho = (rho1 - rho2)/2 grad phi; P = sum f + cs^2/2 u.grad rho */
      double drx = 0.5 * (rho1 - rho2) * m[M_GX * n + k];
      double dry = 0.5 * (rho1 - rho2) * m[M_GY * n + k];
      m[M_FX * n + k] = Fx;
      m[M_FY * n + k] = Fy;
      m[M_RHO * n + k] = rho;
      m[M_UX * n + k] = ux;
      m[M_UY * n + k] = uy;
      double P = sf + (ux * drx + uy * dry) / 6.0;
      m[M_P * n + k] = P;
      /* hydrodynamic pressure p_h from the generalised pressure of each
       * form: P_stf-2 = p_h (Eq. SF2), Eq. P3456 for CPF/PF, P_csf = p_h,
       * and P_stf-1 = p_h - kappa |grad phi|^2.  Eq. SF1 prints the STF-1
       * term with a plus sign, but F_stf-1 = F_stf-2 - kappa grad |grad phi|^2
       * (Eqs. SF1, SF2) and the same momentum equation for both forms fix
       * the minus sign, which is also the one Eq. P3456 implies through
       * Eq. identity (P_pf-1 - P_stf-1 = kappa |grad phi|^2 / 2). */
      double g2 = m[M_GX * n + k] * m[M_GX * n + k] + m[M_GY * n + k] * m[M_GY * n + k];
      double f0 = beta * (1.0 - ph * ph) * (1.0 - ph * ph);
      double muk = m[M_MU * n + k], Lk = m[M_LAP * n + k];
      double ph_p = P;
      switch (form) {
        case STF1: ph_p = P + kap * g2; break;
        case CPF1: ph_p = P - f0 + ph * muk + 0.5 * kap * g2; break;
        case CPF2: ph_p = P - f0 + 0.5 * kap * g2; break;
        case PF1: ph_p = P + 0.5 * kap * g2; break;
        case PF2: ph_p = P - kap * ph * Lk + 0.5 * kap * g2; break;
        default: break;
      }
      m[M_PH * n + k] = ph_p;
      m[M_PUX * n + k] = ph * ux;
      m[M_PUY * n + k] = ph * uy;
      m[M_TAUF * n + k] = tauf;
    }

  /* 6. div(phi u) and d_t(phi u).  Wall ghost of phi u: phi (2 u_w - u) of
   * the mirrored node, built explicitly here. */
  const double* pux = m + M_PUX * n;
  const double* puy = m + M_PUY * n;
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t k = (size_t)y * nx + x;
      double s = 0.0;
      for (int i = 1; i < NQ; ++i) {
        int xx = wrapx(&g, x + ex[i]);
        int yy = y + ey[i];
        double vx, vy;
        if (!wall) {
          yy = (yy + ny) % ny;
          vx = pux[(size_t)yy * nx + xx];
          vy = puy[(size_t)yy * nx + xx];
        } else if (yy < 0 || yy >= ny) {
          int ym = yy < 0 ? 0 : ny - 1; /* mirror of row -1 is row 0 */
          double uw = yy < 0 ? p[P_UWB] : p[P_UWT];
          size_t km = (size_t)ym * nx + xx;
          double pm = phi[km];
          vx = pm * (2.0 * uw - m[M_UX * n + km]);
          vy = pm * (0.0 - m[M_UY * n + km]);
        } else {
          vx = pux[(size_t)yy * nx + xx];
          vy = puy[(size_t)yy * nx + xx];
        }
        s += wq[i] * (ex[i] * vx + ey[i] * vy);
      }
      m[M_DIV * n + k] = 3.0 * s;
      if (first) {
        m[M_DTX * n + k] = 0.0;
        m[M_DTY * n + k] = 0.0;
      } else {
        m[M_DTX * n + k] = pux[k] - phiu_prev[k];
        m[M_DTY * n + k] = puy[k] - phiu_prev[n + k];
      }
    }
  free(xf);
}

/* --------------------------------------------------------------------- */
/* one full step                                                          */
/* --------------------------------------------------------------------- */

/* Advance (f, h, phiu_prev) by nsteps steps in place.  f, h are the
 * pre-collision populations at time t; on return they are those at t+nsteps.
 * `first` marks that the first of these steps is the first of the run. */
static void step_px(const double* p, int nx, int ny, int wall, double* f, double* h,
                    double* phiu_prev, int nsteps, int first) {
  Grid g = {nx, ny, wall};
  size_t n = (size_t)nx * ny;
  double* m = (double*)malloc(sizeof(double) * M_NFIELDS * n);
  double* fp = (double*)malloc(sizeof(double) * NQ * n);
  double* hp = (double*)malloc(sizeof(double) * NQ * n);
  double tau_h = p[P_TAUH];
  double eta = p[P_M] / ((tau_h - 0.5) / 3.0); /* M = cs^2 eta (tau_h - 1/2) */

  for (int step = 0; step < nsteps; ++step) {
    macro_px(p, nx, ny, wall, f, h, phiu_prev, first && step == 0, m);

    /* 7. collision */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        size_t k = (size_t)y * nx + x;
        double ux = m[M_UX * n + k], uy = m[M_UY * n + k];
        double rho = m[M_RHO * n + k], P = m[M_P * n + k];
        double tauf = m[M_TAUF * n + k];
        double drx = 0.5 * (p[P_RHO1] - p[P_RHO2]) * m[M_GX * n + k];
        double dry = 0.5 * (p[P_RHO1] - p[P_RHO2]) * m[M_GY * n + k];
        double feq[NQ], Fi[NQ], heq[NQ], Hi[NQ];
        orc_feq(P, rho, ux, uy, feq);
        orc_fforce(ux, uy, m[M_FX * n + k], m[M_FY * n + k], drx, dry, Fi);
        orc_heq(m[M_PHI * n + k], m[M_MU * n + k], eta, ux, uy, heq);
        orc_hsource(tau_h, m[M_DIV * n + k], m[M_DTX * n + k], m[M_DTY * n + k], Hi);
        for (int i = 0; i < NQ; ++i) {
          double fi = f[i * n + k];
          double hi = h[i * n + k];
          fp[i * n + k] = fi - (fi - feq[i]) / tauf + (1.0 - 0.5 / tauf) * Fi[i];
          hp[i * n + k] = hi - (hi - heq[i]) / tau_h + (1.0 - 0.5 / tau_h) * Hi[i];
        }
      }

    /* 8. streaming with periodic wrap or half-way bounce-back at y walls */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < nx; ++x) {
        size_t k = (size_t)y * nx + x;
        for (int i = 0; i < NQ; ++i) {
          int xt = wrapx(&g, x + ex[i]);
          int yt = y + ey[i];
          if (!wall) {
            yt = (yt + ny) % ny;
          } else if (yt < 0 || yt >= ny) {
            /* the population leaves through a wall: it returns to x in the
             * opposite direction, minus the moving-wall term */
            double uw = yt < 0 ? p[P_UWB] : p[P_UWT];
            double cu = ex[i] * uw; /* c_i . u_w, u_w = (uw, 0) */
            int o = opp[i];
            f[o * n + k] = fp[i * n + k] - 2.0 * wq[i] * m[M_RHO * n + k] * cu;
            h[o * n + k] = hp[i * n + k] - 2.0 * wq[i] * m[M_PHI * n + k] * 3.0 * cu;
            continue;
          }
          size_t kt = (size_t)yt * nx + xt;
          f[i * n + kt] = fp[i * n + k];
          h[i * n + kt] = hp[i * n + k];
        }
      }

    /* 9. keep phi u for the next time derivative */
    memcpy(phiu_prev, m + M_PUX * n, sizeof(double) * n);
    memcpy(phiu_prev + n, m + M_PUY * n, sizeof(double) * n);
  }
  free(m);
  free(fp);
  free(hp);
}

/* Initial state (phi0 given, u = 0, P = 0): f = f^eq(0, rho, 0) = 0 and
 * h = h^eq(phi0, mu0, 0) with mu0 from the chemical potential of phi0. */
static void init_px(const double* p, int nx, int ny, int wall, const double* phi0,
                    double* f, double* h, double* phiu_prev) {
  Grid g = {nx, ny, wall};
  size_t n = (size_t)nx * ny;
  double beta = beta_of(p), kap = kappa_of(p);
  double eta = p[P_M] / ((p[P_TAUH] - 0.5) / 3.0);
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t k = (size_t)y * nx + x;
      double ph = phi0[k];
      double L = ics_lap_node(&g, phi0, x, y);
      double mu = 4.0 * beta * ph * (ph * ph - 1.0) - kap * L;
      double heq[NQ];
      orc_heq(ph, mu, eta, 0.0, 0.0, heq);
      for (int i = 0; i < NQ; ++i) {
        f[i * n + k] = 0.0;
        h[i * n + k] = heq[i];
      }
      phiu_prev[k] = 0.0;
      phiu_prev[n + k] = 0.0;
    }
}

/* Stand-alone central-scheme operators on a periodic or walled field, for
 * the stencil tests: out = [gx | gy | lap], each [ny][nx]. */
static void ics_px(int nx, int ny, int wall, const double* a, double* out) {
  Grid g = {nx, ny, wall};
  size_t n = (size_t)nx * ny;
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < nx; ++x) {
      size_t k = (size_t)y * nx + x;
      double gx, gy;
      ics_grad_node(&g, a, 1.0, x, y, &gx, &gy);
      out[k] = gx;
      out[n + k] = gy;
      out[2 * n + k] = ics_lap_node(&g, a, x, y);
    }
}

/* --------------------------------------------------------------------- */
/* free-slip walls at x = -1/2 and x = nx - 1/2 (bit 1 of `wall`)          */
/* --------------------------------------------------------------------- */
/* A free-slip (specular) wall is a plane of mirror symmetry.  A domain with
 * such walls at x = -1/2 and nx - 1/2 is therefore one half of the periodic
 * domain of width 2 nx whose state is mirror-symmetric about x = nx - 1/2:
 * node x of the other half is 2 nx - 1 - x, population i there is the mirror
 * population (c_x reversed) of the node it mirrors, and x-odd fields (the x
 * component of phi u) change sign.  The oracle is that definition written
 * out: every step builds the symmetric doubled state from this half, runs one
 * periodic-x step on it and keeps this half.  The doubled domain is symmetric
 * only when the forcing is: gravity along x and wall motion along x (both odd
 * under the mirror) must be zero, which the caller checks. */
static const int mirx[NQ] = {0, 3, 2, 1, 4, 6, 5, 8, 7};

static void dbl_pops(int nx, int ny, const double* a, double* d) {
  size_t n = (size_t)nx * ny, n2 = 2 * n;
  for (int i = 0; i < NQ; ++i)
    for (int y = 0; y < ny; ++y)
      for (int x = 0; x < 2 * nx; ++x)
        d[i * n2 + (size_t)y * 2 * nx + x] =
            x < nx ? a[i * n + (size_t)y * nx + x]
                   : a[mirx[i] * n + (size_t)y * nx + (2 * nx - 1 - x)];
}
static void dbl_field(int nx, int ny, const double* a, double* d, double sign) {
  for (int y = 0; y < ny; ++y)
    for (int x = 0; x < 2 * nx; ++x)
      d[(size_t)y * 2 * nx + x] =
          x < nx ? a[(size_t)y * nx + x] : sign * a[(size_t)y * nx + (2 * nx - 1 - x)];
}
static void half_planes(int nx, int ny, int planes, const double* d, double* a) {
  size_t n = (size_t)nx * ny, n2 = 2 * n;
  for (int i = 0; i < planes; ++i)
    for (int y = 0; y < ny; ++y)
      memcpy(a + i * n + (size_t)y * nx, d + i * n2 + (size_t)y * 2 * nx, sizeof(double) * nx);
}

void orc_macro(const double* p, int nx, int ny, int wall, const double* f, const double* h,
               const double* phiu_prev, int first, double* out) {
  if (!(wall & 2)) {
    macro_px(p, nx, ny, wall, f, h, phiu_prev, first, out);
    return;
  }
  size_t n2 = (size_t)2 * nx * ny;
  double* fd = (double*)malloc(sizeof(double) * NQ * n2);
  double* hd = (double*)malloc(sizeof(double) * NQ * n2);
  double* qd = (double*)malloc(sizeof(double) * 2 * n2);
  double* od = (double*)malloc(sizeof(double) * M_NFIELDS * n2);
  dbl_pops(nx, ny, f, fd);
  dbl_pops(nx, ny, h, hd);
  dbl_field(nx, ny, phiu_prev, qd, -1.0);
  dbl_field(nx, ny, phiu_prev + (size_t)nx * ny, qd + n2, 1.0);
  macro_px(p, 2 * nx, ny, wall & 1, fd, hd, qd, first, od);
  half_planes(nx, ny, M_NFIELDS, od, out);
  free(fd);
  free(hd);
  free(qd);
  free(od);
}

void orc_step(const double* p, int nx, int ny, int wall, double* f, double* h,
              double* phiu_prev, int nsteps, int first) {
  if (!(wall & 2)) {
    step_px(p, nx, ny, wall, f, h, phiu_prev, nsteps, first);
    return;
  }
  size_t n = (size_t)nx * ny, n2 = 2 * n;
  double* fd = (double*)malloc(sizeof(double) * NQ * n2);
  double* hd = (double*)malloc(sizeof(double) * NQ * n2);
  double* qd = (double*)malloc(sizeof(double) * 2 * n2);
  for (int s = 0; s < nsteps; ++s) {
    dbl_pops(nx, ny, f, fd);
    dbl_pops(nx, ny, h, hd);
    dbl_field(nx, ny, phiu_prev, qd, -1.0);
    dbl_field(nx, ny, phiu_prev + n, qd + n2, 1.0);
    step_px(p, 2 * nx, ny, wall & 1, fd, hd, qd, 1, first && s == 0);
    half_planes(nx, ny, NQ, fd, f);
    half_planes(nx, ny, NQ, hd, h);
    half_planes(nx, ny, 2, qd, phiu_prev);
  }
  free(fd);
  free(hd);
  free(qd);
}

void orc_init(const double* p, int nx, int ny, int wall, const double* phi0, double* f,
              double* h, double* phiu_prev) {
  if (!(wall & 2)) {
    init_px(p, nx, ny, wall, phi0, f, h, phiu_prev);
    return;
  }
  size_t n2 = (size_t)2 * nx * ny;
  double* pd = (double*)malloc(sizeof(double) * n2);
  double* fd = (double*)malloc(sizeof(double) * NQ * n2);
  double* hd = (double*)malloc(sizeof(double) * NQ * n2);
  double* qd = (double*)malloc(sizeof(double) * 2 * n2);
  dbl_field(nx, ny, phi0, pd, 1.0);
  init_px(p, 2 * nx, ny, wall & 1, pd, fd, hd, qd);
  half_planes(nx, ny, NQ, fd, f);
  half_planes(nx, ny, NQ, hd, h);
  half_planes(nx, ny, 2, qd, phiu_prev);
  free(pd);
  free(fd);
  free(hd);
  free(qd);
}

void orc_ics(int nx, int ny, int wall, const double* a, double* out) {
  if (!(wall & 2)) {
    ics_px(nx, ny, wall, a, out);
    return;
  }
  size_t n2 = (size_t)2 * nx * ny;
  double* ad = (double*)malloc(sizeof(double) * n2);
  double* od = (double*)malloc(sizeof(double) * 3 * n2);
  dbl_field(nx, ny, a, ad, 1.0);
  ics_px(2 * nx, ny, wall & 1, ad, od);
  half_planes(nx, ny, 3, od, out);
  free(ad);
  free(od);
}

int orc_nfields(void) { return M_NFIELDS; }
int orc_npar(void) { return P_NPAR; }

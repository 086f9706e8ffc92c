// Hand-written discrete adjoint of one coupled step (Sec. 3 of Zhang, Liang &
// Guo, arXiv 2012.14729), FP32 fields with FP64 parameter accumulators.
//
// The reverse of a step runs as a sequence of one-thread-per-node kernels:
// first the step's intermediates are recomputed from the stored pre-collision
// populations at time t (phi, moments, grad phi, lap phi, mu, the force of the
// selected form, rho, u, P, phi u, div(phi u), d_t(phi u)), then the adjoints
// flow back through the collision and streaming (with the bounce-back terms),
// div(phi u), the macroscopic relations, the force, the chemical potential and
// the central-scheme stencils.  The transpose of each stencil is a gather over
// the nodes whose stencil reads a node, directly or through a wall ghost
// (mirror rule with the field's parity) or the periodic seam.  Parameter
// gradients d/d(4 beta), d/d kappa, d/d eta and the direct d/d sigma of CSF-2
// are summed per block in double precision and added to four accumulators.
#include "lattice.cuh"

namespace pflbm {

namespace {

constexpr int kAB = 128;  // threads per block (one row segment)

using Geo = AdjGeo;

__device__ __forceinline__ int wx(const Geo& g, int x) {
  return x < 0 ? x + g.nx : (x >= g.nx ? x - g.nx : x);
}

// value of a node field at (x, y) with one ghost row: periodic wrap, or the
// wall mirror ghost (row -1 = row 0, row ny = row ny - 1) times `parity`
__device__ __forceinline__ float at(const float* a, const Geo& g, int x, int y, float parity) {
  x = wx(g, x);
  float s = 1.0f;
  if (y < 0) {
    if (g.wall) { y = 0; s = parity; } else y += g.ny;
  } else if (y >= g.ny) {
    if (g.wall) { y = g.ny - 1; s = parity; } else y -= g.ny;
  }
  return s * a[y * g.nx + x];
}

// Eq. ICS-1st: d/d(axis) of a node field read with `parity` at its ghosts
__device__ __forceinline__ float dfw(const float* a, const Geo& g, int x, int y, int axis,
                                     float parity) {
  float s = 0.0f;
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const int c = axis == 0 ? qcx(i) : qcy(i);
    if (c != 0) s += (3.0f * qw(i) * c) * at(a, g, x + qcx(i), y + qcy(i), parity);
  }
  return s;
}

// Eq. ICS-sec (even field)
__device__ __forceinline__ float lapfw(const float* a, const Geo& g, int x, int y) {
  const float c = a[y * g.nx + x];
  float s = 0.0f;
#pragma unroll
  for (int i = 1; i < 9; ++i) s += (6.0f * qw(i)) * (at(a, g, x + qcx(i), y + qcy(i), 1.0f) - c);
  return s;
}

// Transpose of dfw: sum over the nodes x' whose stencil reads node (x, y),
// directly or through a ghost, of coef_i * b(x').  `wcoef` selects the
// weights: 3 w_i c_i,axis (derivative) or 6 w_i (Laplacian neighbour part).
template <bool LAP>
__device__ __forceinline__ float stencil_T(const float* b, const Geo& g, int x, int y, int axis,
                                           float parity) {
  float s = 0.0f;
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const int c = LAP ? 1 : (axis == 0 ? qcx(i) : qcy(i));
    if (c == 0) continue;
    const float coef = LAP ? 6.0f * qw(i) : 3.0f * qw(i) * c;
    const int xs = wx(g, x - qcx(i));
    int ys = y - qcy(i);
    if (g.wall) {
      if (ys >= 0 && ys < g.ny) s += coef * b[ys * g.nx + xs];
      // node (xs, y) on a wall row reads the ghost that folds onto (x, y)
      if (y == 0 && qcy(i) == -1) s += parity * coef * b[xs];
      if (y == g.ny - 1 && qcy(i) == 1) s += parity * coef * b[(g.ny - 1) * g.nx + xs];
    } else {
      ys = ys < 0 ? ys + g.ny : (ys >= g.ny ? ys - g.ny : ys);
      s += coef * b[ys * g.nx + xs];
    }
  }
  if (LAP) s -= (10.0f / 3.0f) * b[y * g.nx + x];  // - sum_i 6 w_i b(x)
  return s;
}

// FP64 block sum of up to 4 per-thread contributions into acc[0..3]
__device__ __forceinline__ void acc_add(double* acc, double v0, double v1, double v2, double v3) {
  __shared__ double red[kAB / 32][4];
  double v[4] = {v0, v1, v2, v3};
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 4; ++k) red[w][k] = v[k];
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int j = 0; j < kAB / 32; ++j) s += red[j][threadIdx.x];
    if (s != 0.0) atomicAdd(&acc[threadIdx.x], s);
  }
}

}  // namespace

// Field slots of the adjoint scratch, each [ny][nx] float32.
enum AdjField {
  // forward intermediates
  A_PHI, A_S, A_JX, A_JY, A_GX, A_GY, A_L, A_MU, A_E0, A_E1, A_E2, A_FSX, A_FSY, A_RHO, A_FX,
  A_FY, A_UX, A_UY, A_PR, A_PX, A_PY, A_DIV, A_DTX, A_DTY, A_OM,
  // adjoints
  B_PHI, B_S, B_JX, B_JY, B_GX, B_GY, B_L, B_MU, B_RHO, B_UX, B_UY, B_P, B_FX, B_FY, B_DIV, B_DTX,
  B_DTY, B_PX, B_PY, B_W0, B_W1, B_W2,
  A_NFIELDS
};

#define ADJ_NODE                                              \
  const int x = blockIdx.x * kAB + threadIdx.x, y = blockIdx.y; \
  const int n = A.g.nx * A.g.ny;                              \
  const bool live = x < A.g.nx;                               \
  const int k = y * A.g.nx + (live ? x : 0);                  \
  float* F = A.F;                                             \
  (void)n;
#define FLD(s) (F + (size_t)(s) * n)

// ---- forward recomputation ----------------------------------------------------
__global__ void k_adj_fwd_moments(const AdjArgs A) {
  ADJ_NODE
  if (!live) return;
  float phi = 0.0f, S = 0.0f, jx = 0.0f, jy = 0.0f;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const float fi = A.fpop[i * n + k];
    phi += A.hpop[i * n + k];
    S += fi;
    jx += qcx(i) * fi;
    jy += qcy(i) * fi;
  }
  FLD(A_PHI)[k] = phi;
  FLD(A_S)[k] = S;
  FLD(A_JX)[k] = jx;
  FLD(A_JY)[k] = jy;
}

__global__ void k_adj_fwd_grad(const AdjArgs A) {
  ADJ_NODE
  if (!live) return;
  const float* phi = FLD(A_PHI);
  const float gx = dfw(phi, A.g, x, y, 0, 1.0f), gy = dfw(phi, A.g, x, y, 1, 1.0f);
  const float L = lapfw(phi, A.g, x, y);
  const float ph = phi[k];
  FLD(A_GX)[k] = gx;
  FLD(A_GY)[k] = gy;
  FLD(A_L)[k] = L;
  FLD(A_MU)[k] = A.p.beta4 * ph * ((ph - 1.0f) * (ph + 1.0f)) - A.p.kappa * L;
  // level-1 fields of the form read by the force stencils
  if (A.form == kSTF1 || A.form == kSTF2) {
    FLD(A_E0)[k] = gx * gx;
    FLD(A_E1)[k] = gx * gy;
    FLD(A_E2)[k] = gy * gy;
  } else if (A.form == kCSF1 || A.form == kCSF2) {
    const float r = sqrtf(gx * gx + gy * gy + A.p.eps2);
    FLD(A_E0)[k] = gx / r;
    FLD(A_E1)[k] = gy / r;
    FLD(A_E2)[k] = r;
  }
}

__global__ void k_adj_fwd_force(const AdjArgs A) {
  ADJ_NODE
  if (!live) return;
  const Phys& P = A.p;
  const float gx = FLD(A_GX)[k], gy = FLD(A_GY)[k], phi = FLD(A_PHI)[k];
  float fx = 0.0f, fy = 0.0f, aux0 = 0.0f, aux1 = 0.0f;
  switch (A.form) {
    case kSTF1:
    case kSTF2: {
      // F = kappa (aux0, aux1): -div(grad phi (x) grad phi) [+ grad |grad phi|^2]
      aux0 = -(dfw(FLD(A_E0), A.g, x, y, 0, 1.0f) + dfw(FLD(A_E1), A.g, x, y, 1, -1.0f));
      aux1 = -(dfw(FLD(A_E1), A.g, x, y, 0, -1.0f) + dfw(FLD(A_E2), A.g, x, y, 1, 1.0f));
      if (A.form == kSTF2) {
        aux0 += dfw(FLD(A_E0), A.g, x, y, 0, 1.0f) + dfw(FLD(A_E2), A.g, x, y, 0, 1.0f);
        aux1 += dfw(FLD(A_E0), A.g, x, y, 1, 1.0f) + dfw(FLD(A_E2), A.g, x, y, 1, 1.0f);
      }
      fx = P.kappa * aux0;
      fy = P.kappa * aux1;
      break;
    }
    case kCPF1:
      aux0 = dfw(FLD(A_MU), A.g, x, y, 0, 1.0f);
      aux1 = dfw(FLD(A_MU), A.g, x, y, 1, 1.0f);
      fx = -phi * aux0;
      fy = -phi * aux1;
      break;
    case kCPF2:
      fx = FLD(A_MU)[k] * gx;
      fy = FLD(A_MU)[k] * gy;
      break;
    case kPF1:
      fx = -P.kappa * gx * FLD(A_L)[k];
      fy = -P.kappa * gy * FLD(A_L)[k];
      break;
    case kPF2:
      aux0 = dfw(FLD(A_L), A.g, x, y, 0, 1.0f);
      aux1 = dfw(FLD(A_L), A.g, x, y, 1, 1.0f);
      fx = P.kappa * phi * aux0;
      fy = P.kappa * phi * aux1;
      break;
    default: {  // CSF: aux0 = div n
      aux0 = dfw(FLD(A_E0), A.g, x, y, 0, 1.0f) + dfw(FLD(A_E1), A.g, x, y, 1, -1.0f);
      const float coef = A.form == kCSF1 ? -P.kappa * sqrtf(gx * gx + gy * gy) * aux0
                                         : -P.half_sigma * aux0;
      fx = coef * gx;
      fy = coef * gy;
    }
  }
  FLD(A_FSX)[k] = fx;
  FLD(A_FSY)[k] = fy;
  // auxiliary values of the force kept for its adjoint (W slots are free now)
  FLD(B_W0)[k] = aux0;
  FLD(B_W1)[k] = aux1;
}

__global__ void k_adj_fwd_macro(const AdjArgs A) {
  ADJ_NODE
  if (!live) return;
  const Phys& P = A.p;
  const float phi = FLD(A_PHI)[k];
  const float rho = P.rho_mid + P.drho_half * phi;
  const float Fx = FLD(A_FSX)[k] + (rho - P.rho0) * P.gx;
  const float Fy = FLD(A_FSY)[k] + (rho - P.rho0) * P.gy;
  const float ux = (3.0f * FLD(A_JX)[k] + 0.5f * Fx) / rho;
  const float uy = (3.0f * FLD(A_JY)[k] + 0.5f * Fy) / rho;
  const float Rx = P.drho_half * FLD(A_GX)[k], Ry = P.drho_half * FLD(A_GY)[k];
  FLD(A_RHO)[k] = rho;
  FLD(A_FX)[k] = Fx;
  FLD(A_FY)[k] = Fy;
  FLD(A_UX)[k] = ux;
  FLD(A_UY)[k] = uy;
  FLD(A_PR)[k] = FLD(A_S)[k] + (ux * Rx + uy * Ry) / 6.0f;
  FLD(A_PX)[k] = phi * ux;
  FLD(A_PY)[k] = phi * uy;
  const float mv = P.mu_mid + P.mu_dhalf * phi;
  FLD(A_OM)[k] = 1.0f / (0.5f + 3.0f * mv / rho);
}

// div(phi u) with the wall ghost phi (2 u_w - u) of the mirrored node
__device__ __forceinline__ float p_ghost(const AdjArgs& A, const float* F, int n, int x, int y,
                                         int comp) {
  const float* px = FLD(A_PX);
  const float* py = FLD(A_PY);
  const Geo& g = A.g;
  x = wx(g, x);
  if (y < 0 || y >= g.ny) {
    if (!g.wall) {
      y = y < 0 ? y + g.ny : y - g.ny;
      return (comp == 0 ? px : py)[y * g.nx + x];
    }
    const int ym = y < 0 ? 0 : g.ny - 1;
    const float uw = y < 0 ? A.p.uwb : A.p.uwt;
    const int km = ym * g.nx + x;
    if (comp == 0) return 2.0f * uw * FLD(A_PHI)[km] - px[km];
    return -py[km];
  }
  return (comp == 0 ? px : py)[y * g.nx + x];
}

__global__ void k_adj_fwd_div(const AdjArgs A) {
  ADJ_NODE
  if (!live) return;
  float s = 0.0f;
#pragma unroll
  for (int i = 1; i < 9; ++i)
    s += 3.0f * qw(i) *
         (qcx(i) * p_ghost(A, F, n, x + qcx(i), y + qcy(i), 0) +
          qcy(i) * p_ghost(A, F, n, x + qcx(i), y + qcy(i), 1));
  FLD(A_DIV)[k] = s;
  FLD(A_DTX)[k] = A.first ? 0.0f : FLD(A_PX)[k] - A.q[k];
  FLD(A_DTY)[k] = A.first ? 0.0f : FLD(A_PY)[k] - A.q[n + k];
}

// ---- reverse ---------------------------------------------------------------------
// streaming transpose + collision transpose (+ bounce-back terms)
__global__ void k_adj_collide(const AdjArgs A) {
  ADJ_NODE
  const Phys& P = A.p;
  const Geo& g = A.g;
  double deta = 0.0;
  if (live) {
    const float phi = FLD(A_PHI)[k], rho = FLD(A_RHO)[k], ux = FLD(A_UX)[k], uy = FLD(A_UY)[k];
    const float Fx = FLD(A_FX)[k], Fy = FLD(A_FY)[k], Pr = FLD(A_PR)[k], om = FLD(A_OM)[k];
    const float Rx = P.drho_half * FLD(A_GX)[k], Ry = P.drho_half * FLD(A_GY)[k];
    const float mu = FLD(A_MU)[k];
    const float uu = ux * ux + uy * uy, uF = ux * Fx + uy * Fy, uR = (ux * Rx + uy * Ry) / 3.0f;
    const float tauh = 1.0f / P.inv_tau_h;
    float phib = 0.0f, rhob = 0.0f, uxb = 0.0f, uyb = 0.0f, Pb = 0.0f, Fxb = 0.0f, Fyb = 0.0f;
    float Rxb = 0.0f, Ryb = 0.0f, mub = 0.0f, divb = 0.0f, dtxb = 0.0f, dtyb = 0.0f, omb = 0.0f;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      // adjoint of the post-collision population: pull transpose (push), or
      // the reflected population where x + c_i lies beyond a wall
      const int xn = wx(g, x + qcx(i));
      int yn = y + qcy(i);
      float fpb, hpb;
      if (g.wall && (yn < 0 || yn >= g.ny)) {
        const int o = qopp(i);
        fpb = A.fb_in[o * n + k];
        hpb = A.hb_in[o * n + k];
        const float cu = qcx(i) * (yn < 0 ? P.uwb : P.uwt);
        rhob += -2.0f * qw(i) * cu * fpb;
        phib += -6.0f * qw(i) * cu * hpb;
      } else {
        if (!g.wall) yn = yn < 0 ? yn + g.ny : (yn >= g.ny ? yn - g.ny : yn);
        fpb = A.fb_in[i * n + yn * g.nx + xn];
        hpb = A.hb_in[i * n + yn * g.nx + xn];
      }
      const float cu = qcx(i) * ux + qcy(i) * uy;
      const float s = 3.0f * cu + 4.5f * cu * cu - 1.5f * uu;
      const float feq = qw(i) * (Pr + rho / 3.0f * s);
      const float cF = qcx(i) * Fx + qcy(i) * Fy;
      const float cR = (qcx(i) * Rx + qcy(i) * Ry) / 3.0f;
      const float Fi = qw(i) * ((1.0f + s) * (cF - uF) + s * (cR - uR));
      A.fb_out[i * n + k] = (1.0f - om) * fpb;
      omb += fpb * (-A.fpop[i * n + k] + feq - 0.5f * Fi);
      const float feqb = om * fpb, Fib = (1.0f - 0.5f * om) * fpb;
      Pb += qw(i) * feqb;
      rhob += qw(i) * s / 3.0f * feqb;
      float sb = qw(i) * rho / 3.0f * feqb;
      sb += qw(i) * ((cF - uF) + (cR - uR)) * Fib;
      const float k1 = qw(i) * (1.0f + s) * Fib, k2 = qw(i) * s * Fib;
      Fxb += k1 * (qcx(i) - ux);
      Fyb += k1 * (qcy(i) - uy);
      uxb += -k1 * Fx - k2 * Rx / 3.0f;
      uyb += -k1 * Fy - k2 * Ry / 3.0f;
      Rxb += k2 * (qcx(i) - ux) / 3.0f;
      Ryb += k2 * (qcy(i) - uy) / 3.0f;
      uxb += sb * ((3.0f + 9.0f * cu) * qcx(i) - 3.0f * ux);
      uyb += sb * ((3.0f + 9.0f * cu) * qcy(i) - 3.0f * uy);
      // h
      A.hb_out[i * n + k] = (1.0f - P.inv_tau_h) * hpb;
      const float heqb = hpb / tauh, Hb = P.hforce * hpb;
      if (i == 0) {
        phib += heqb;
        mub += (qw(0) - 1.0f) * P.eta * heqb;
        deta += (double)((qw(0) - 1.0f) * mu * heqb);
      } else {
        mub += qw(i) * P.eta * heqb;
        deta += (double)(qw(i) * mu * heqb);
        phib += 3.0f * qw(i) * cu * heqb;
        uxb += 3.0f * qw(i) * phi * qcx(i) * heqb;
        uyb += 3.0f * qw(i) * phi * qcy(i) * heqb;
      }
      divb += (i == 0 ? qw(0) - 1.0f : qw(i)) * P.acoef * Hb;
      dtxb += 3.0f * qw(i) * qcx(i) * Hb;
      dtyb += 3.0f * qw(i) * qcy(i) * Hb;
    }
    // omega = 1/tau_f, tau_f = 1/2 + 3 mu_v / rho
    const float mv = P.mu_mid + P.mu_dhalf * phi;
    const float taub = -om * om * omb;
    phib += P.mu_dhalf * (3.0f / rho * taub);
    rhob += -3.0f * mv / (rho * rho) * taub;
    FLD(B_PHI)[k] = phib;
    FLD(B_RHO)[k] = rhob;
    FLD(B_UX)[k] = uxb;
    FLD(B_UY)[k] = uyb;
    FLD(B_P)[k] = Pb;
    FLD(B_FX)[k] = Fxb;
    FLD(B_FY)[k] = Fyb;
    FLD(B_GX)[k] = P.drho_half * Rxb;  // R = (rho1 - rho2)/2 grad phi
    FLD(B_GY)[k] = P.drho_half * Ryb;
    FLD(B_MU)[k] = mub;
    FLD(B_DIV)[k] = divb;
    FLD(B_DTX)[k] = dtxb;
    FLD(B_DTY)[k] = dtyb;
  }
  acc_add(A.acc, 0.0, 0.0, deta, 0.0);
}

// adjoint of div(phi u) and of d_t(phi u) = p - q, plus the incoming adjoint of (phi u)^t
__global__ void k_adj_div(const AdjArgs A) {
  ADJ_NODE
  if (!live) return;
  const Geo& g = A.g;
  const float* divb = FLD(B_DIV);
  // p_x is read as parity -1 with an additive 2 u_w phi at the wall ghosts,
  // p_y with parity -1; periodic wraps
  float pxb = stencil_T<false>(divb, g, x, y, 0, -1.0f);
  float pyb = stencil_T<false>(divb, g, x, y, 1, -1.0f);
  if (g.wall && (y == 0 || y == g.ny - 1)) {
    // ghost adjoint of p_x at (x, -1) or (x, ny): nodes of this row whose
    // stencil reads it; its 2 u_w phi(x, row) part goes to phi
    const int cyw = y == 0 ? -1 : 1;
    float ga = 0.0f;
#pragma unroll
    for (int i = 1; i < 9; ++i)
      if (qcy(i) == cyw) ga += 3.0f * qw(i) * qcx(i) * divb[y * g.nx + wx(g, x - qcx(i))];
    FLD(B_PHI)[k] += 2.0f * (y == 0 ? A.p.uwb : A.p.uwt) * ga;
  }
  pxb += A.qb_in[k];
  pyb += A.qb_in[n + k];
  if (!A.first) {
    pxb += FLD(B_DTX)[k];
    pyb += FLD(B_DTY)[k];
    A.qb_out[k] = -FLD(B_DTX)[k];
    A.qb_out[n + k] = -FLD(B_DTY)[k];
  } else {
    A.qb_out[k] = 0.0f;
    A.qb_out[n + k] = 0.0f;
  }
  FLD(B_PX)[k] = pxb;
  FLD(B_PY)[k] = pyb;
}

// p = phi u, P = S + u.R/6, u = (3 j + F/2)/rho, F = F_sf + (rho - rho0) g, rho(phi)
__global__ void k_adj_macro(const AdjArgs A) {
  ADJ_NODE
  if (!live) return;
  const Phys& P = A.p;
  const float phi = FLD(A_PHI)[k], rho = FLD(A_RHO)[k], ux = FLD(A_UX)[k], uy = FLD(A_UY)[k];
  const float Rx = P.drho_half * FLD(A_GX)[k], Ry = P.drho_half * FLD(A_GY)[k];
  const float pxb = FLD(B_PX)[k], pyb = FLD(B_PY)[k], Pb = FLD(B_P)[k];
  float phib = FLD(B_PHI)[k] + pxb * ux + pyb * uy;
  float uxb = FLD(B_UX)[k] + phi * pxb + Rx / 6.0f * Pb;
  float uyb = FLD(B_UY)[k] + phi * pyb + Ry / 6.0f * Pb;
  float Gxb = FLD(B_GX)[k] + P.drho_half * (ux / 6.0f * Pb);
  float Gyb = FLD(B_GY)[k] + P.drho_half * (uy / 6.0f * Pb);
  FLD(B_S)[k] = Pb;
  FLD(B_JX)[k] = 3.0f * uxb / rho;
  FLD(B_JY)[k] = 3.0f * uyb / rho;
  const float Fxb = FLD(B_FX)[k] + 0.5f * uxb / rho;
  const float Fyb = FLD(B_FY)[k] + 0.5f * uyb / rho;
  float rhob = FLD(B_RHO)[k] - (ux * uxb + uy * uyb) / rho;
  rhob += P.gx * Fxb + P.gy * Fyb;
  phib += P.drho_half * rhob;
  FLD(B_PHI)[k] = phib;
  FLD(B_GX)[k] = Gxb;
  FLD(B_GY)[k] = Gyb;
  FLD(B_FX)[k] = Fxb;  // now the adjoint of F_sf
  FLD(B_FY)[k] = Fyb;
}

// pointwise part of the force adjoint; leaves in W0..W2 what the stencil
// transposes need
__global__ void k_adj_force_pt(const AdjArgs A) {
  ADJ_NODE
  const Phys& P = A.p;
  double dk = 0.0, ds = 0.0;
  if (live) {
    const float gx = FLD(A_GX)[k], gy = FLD(A_GY)[k], phi = FLD(A_PHI)[k];
    const float Fxb = FLD(B_FX)[k], Fyb = FLD(B_FY)[k];
    float w0 = 0.0f, w1 = 0.0f, w2 = 0.0f;
    switch (A.form) {
      case kSTF1:
      case kSTF2:
        dk = (double)Fxb * FLD(B_W0)[k] + (double)Fyb * FLD(B_W1)[k];
        break;
      case kCPF1:
        FLD(B_PHI)[k] += -(FLD(B_W0)[k] * Fxb + FLD(B_W1)[k] * Fyb);
        w0 = -phi * Fxb;
        w1 = -phi * Fyb;
        break;
      case kCPF2:
        FLD(B_MU)[k] += gx * Fxb + gy * Fyb;
        FLD(B_GX)[k] += FLD(A_MU)[k] * Fxb;
        FLD(B_GY)[k] += FLD(A_MU)[k] * Fyb;
        break;
      case kPF1: {
        const float L = FLD(A_L)[k];
        FLD(B_GX)[k] += -P.kappa * L * Fxb;
        FLD(B_GY)[k] += -P.kappa * L * Fyb;
        FLD(B_L)[k] = -P.kappa * (gx * Fxb + gy * Fyb);
        dk = -(double)(gx * Fxb + gy * Fyb) * L;
        break;
      }
      case kPF2: {
        const float dlx = FLD(B_W0)[k], dly = FLD(B_W1)[k];
        FLD(B_PHI)[k] += P.kappa * (dlx * Fxb + dly * Fyb);
        dk = (double)phi * (dlx * Fxb + dly * Fyb);
        w0 = P.kappa * phi * Fxb;
        w1 = P.kappa * phi * Fyb;
        break;
      }
      default: {  // CSF
        const float divn = FLD(B_W0)[k];
        const float a = sqrtf(gx * gx + gy * gy);
        const float GF = gx * Fxb + gy * Fyb;
        float divnb;
        if (A.form == kCSF1) {
          FLD(B_GX)[k] += -P.kappa * a * divn * Fxb;
          FLD(B_GY)[k] += -P.kappa * a * divn * Fyb;
          const float ab = -P.kappa * divn * GF;
          divnb = -P.kappa * a * GF;
          dk = -(double)GF * a * divn;
          if (a > 0.0f) {
            FLD(B_GX)[k] += ab * gx / a;
            FLD(B_GY)[k] += ab * gy / a;
          }
        } else {
          FLD(B_GX)[k] += -P.half_sigma * divn * Fxb;
          FLD(B_GY)[k] += -P.half_sigma * divn * Fyb;
          divnb = -P.half_sigma * GF;
          ds = -0.5 * (double)GF * divn;
        }
        w2 = divnb;
      }
    }
    if (A.form != kPF1) FLD(B_L)[k] = 0.0f;
    FLD(B_W0)[k] = w0;
    FLD(B_W1)[k] = w1;
    FLD(B_W2)[k] = w2;
  }
  acc_add(A.acc, 0.0, dk, 0.0, ds);
}

// stencil part of the force adjoint
__global__ void k_adj_force_st(const AdjArgs A) {
  ADJ_NODE
  if (!live) return;
  const Geo& g = A.g;
  const Phys& P = A.p;
  const float gx = FLD(A_GX)[k], gy = FLD(A_GY)[k];
  switch (A.form) {
    case kSTF1:
    case kSTF2: {
      const float* fxb = FLD(B_FX);
      const float* fyb = FLD(B_FY);
      float txx = -P.kappa * stencil_T<false>(fxb, g, x, y, 0, 1.0f);
      const float txy = -P.kappa * (stencil_T<false>(fxb, g, x, y, 1, -1.0f) +
                                    stencil_T<false>(fyb, g, x, y, 0, -1.0f));
      float tyy = -P.kappa * stencil_T<false>(fyb, g, x, y, 1, 1.0f);
      if (A.form == kSTF2) {
        const float g2b = P.kappa * (stencil_T<false>(fxb, g, x, y, 0, 1.0f) +
                                     stencil_T<false>(fyb, g, x, y, 1, 1.0f));
        txx += g2b;
        tyy += g2b;
      }
      FLD(B_GX)[k] += 2.0f * gx * txx + gy * txy;
      FLD(B_GY)[k] += gx * txy + 2.0f * gy * tyy;
      break;
    }
    case kCPF1:
      FLD(B_MU)[k] += stencil_T<false>(FLD(B_W0), g, x, y, 0, 1.0f) +
                      stencil_T<false>(FLD(B_W1), g, x, y, 1, 1.0f);
      break;
    case kPF2:
      FLD(B_L)[k] += stencil_T<false>(FLD(B_W0), g, x, y, 0, 1.0f) +
                     stencil_T<false>(FLD(B_W1), g, x, y, 1, 1.0f);
      break;
    case kCSF1:
    case kCSF2: {
      const float* divnb = FLD(B_W2);
      const float nxb = stencil_T<false>(divnb, g, x, y, 0, 1.0f);
      const float nyb = stencil_T<false>(divnb, g, x, y, 1, -1.0f);
      const float r = FLD(A_E2)[k];
      const float gn = gx * nxb + gy * nyb;
      FLD(B_GX)[k] += nxb / r - gx * gn / (r * r * r);
      FLD(B_GY)[k] += nyb / r - gy * gn / (r * r * r);
      break;
    }
    default:
      break;
  }
}

// mu = 4 beta phi (phi^2 - 1) - kappa lap phi
__global__ void k_adj_mu(const AdjArgs A) {
  ADJ_NODE
  double db = 0.0, dk = 0.0;
  if (live) {
    const float phi = FLD(A_PHI)[k], mub = FLD(B_MU)[k];
    FLD(B_PHI)[k] += A.p.beta4 * (3.0f * phi * phi - 1.0f) * mub;
    FLD(B_L)[k] += -A.p.kappa * mub;
    db = (double)phi * (phi * phi - 1.0f) * mub;
    dk = -(double)FLD(A_L)[k] * mub;
  }
  acc_add(A.acc, db, dk, 0.0, 0.0);
}

// grad phi, lap phi -> phi; then phi = sum h, S = sum f, j = sum c f
__global__ void k_adj_finish(const AdjArgs A) {
  ADJ_NODE
  if (!live) return;
  const Geo& g = A.g;
  const float phib = FLD(B_PHI)[k] + stencil_T<false>(FLD(B_GX), g, x, y, 0, 1.0f) +
                     stencil_T<false>(FLD(B_GY), g, x, y, 1, 1.0f) +
                     stencil_T<true>(FLD(B_L), g, x, y, 0, 1.0f);
  const float Sb = FLD(B_S)[k], jxb = FLD(B_JX)[k], jyb = FLD(B_JY)[k];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    A.hb_out[i * n + k] += phib;
    A.fb_out[i * n + k] += Sb + qcx(i) * jxb + qcy(i) * jyb;
  }
}

// Reverse of one step: adjoint state (fb_in, hb_in, qb_in) at t + 1 ->
// (fb_out, hb_out, qb_out) at t, with the forward state (fpop, hpop, q) at t.
cudaError_t launch_adjoint_step(const AdjArgs& A, cudaStream_t s) {
  const dim3 grid((A.g.nx + kAB - 1) / kAB, A.g.ny);
  k_adj_fwd_moments<<<grid, kAB, 0, s>>>(A);
  k_adj_fwd_grad<<<grid, kAB, 0, s>>>(A);
  k_adj_fwd_force<<<grid, kAB, 0, s>>>(A);
  k_adj_fwd_macro<<<grid, kAB, 0, s>>>(A);
  k_adj_fwd_div<<<grid, kAB, 0, s>>>(A);
  k_adj_collide<<<grid, kAB, 0, s>>>(A);
  k_adj_div<<<grid, kAB, 0, s>>>(A);
  k_adj_macro<<<grid, kAB, 0, s>>>(A);
  k_adj_force_pt<<<grid, kAB, 0, s>>>(A);
  k_adj_force_st<<<grid, kAB, 0, s>>>(A);
  k_adj_mu<<<grid, kAB, 0, s>>>(A);
  k_adj_finish<<<grid, kAB, 0, s>>>(A);
  return cudaGetLastError();
}

// ---- initial state: h = h^eq(phi0, mu0, 0), f = 0 ------------------------------
// phi0 -> mu0 (grad kernel on phi0 in A_PHI); then phi0 adjoint from hb_in.
__global__ void k_adj_init_pt(const AdjArgs A) {
  ADJ_NODE
  double db = 0.0, dk = 0.0, de = 0.0;
  if (live) {
    const Phys& P = A.p;
    const float phi = FLD(A_PHI)[k], mu = FLD(A_MU)[k];
    float hsum = (qw(0) - 1.0f) * A.hb_in[k];
#pragma unroll
    for (int i = 1; i < 9; ++i) hsum += qw(i) * A.hb_in[i * n + k];
    const float mub = P.eta * hsum;
    de = (double)mu * hsum;
    db = (double)phi * (phi * phi - 1.0f) * mub;
    dk = -(double)FLD(A_L)[k] * mub;
    FLD(B_PHI)[k] = A.hb_in[k] + P.beta4 * (3.0f * phi * phi - 1.0f) * mub;
    FLD(B_L)[k] = -P.kappa * mub;
  }
  acc_add(A.acc, db, dk, de, 0.0);
}

__global__ void k_adj_init_out(const AdjArgs A, float* dphi0) {
  ADJ_NODE
  if (!live) return;
  dphi0[k] = FLD(B_PHI)[k] + stencil_T<true>(FLD(B_L), A.g, x, y, 0, 1.0f);
}

cudaError_t launch_adjoint_init(const AdjArgs& A, const float* phi0, float* dphi0,
                                cudaStream_t s) {
  const dim3 grid((A.g.nx + kAB - 1) / kAB, A.g.ny);
  const size_t n = (size_t)A.g.nx * A.g.ny;
  cudaError_t e = cudaMemcpyAsync(A.F + (size_t)A_PHI * n, phi0, n * 4,
                                  cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return e;
  AdjArgs B = A;
  B.form = kPF1;  // the grad kernel's level-1 extras are not needed here
  k_adj_fwd_grad<<<grid, kAB, 0, s>>>(B);
  k_adj_init_pt<<<grid, kAB, 0, s>>>(A);
  k_adj_init_out<<<grid, kAB, 0, s>>>(A, dphi0);
  return cudaGetLastError();
}

int adjoint_nfields() { return A_NFIELDS; }

}  // namespace pflbm

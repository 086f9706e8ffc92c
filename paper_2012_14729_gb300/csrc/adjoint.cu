// Hand-written discrete adjoint of one coupled step (Sec. 3 of Zhang, Liang &
// Guo, arXiv 2012.14729), FP32 fields with FP64 parameter accumulators.
//
// The forward intermediates of step t (pulled f, phi, grad phi, lap phi, mu,
// the force, u, P, div(phi u), d_t(phi u)) are recorded by the taping step
// (the fused step kernel with its tape output, step_kernel.cuh).  The reverse
// of the step then runs as two kernels:
//   collide  streaming transpose (push, with the bounce-back terms) and the
//            collision transpose of f and h, one thread per node;
//   tail     on 32 x 8 tiles: the transpose of div(phi u) and d_t(phi u), of
//            the macroscopic relations (u, P, rho) and the pointwise part of
//            the force (tile + 2 ring), the transposes of the force stencils
//            and of the chemical potential (tile + 1 ring), and those of
//            grad phi and lap phi into the adjoint of phi (tile).
// The transpose of each stencil is a gather over the nodes whose stencil reads
// a node, directly or through a wall ghost (mirror rule with the field's
// parity) or the periodic seam.  The adjoints of phi = sum h_i and of S, j
// (sums of f_i) are not spread over the 18 populations here: they stay as
// per-node scalars of the adjoint state, added when the next reverse step
// reads a population.  Parameter gradients d/d(4 beta), d/d kappa, d/d eta and
// the direct d/d sigma of CSF-2 are summed per block in double precision and
// added to four accumulators.
#include "step_kernel.cuh"


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
// IN: the node and the nodes its transpose reads lie inside the domain, off
// the wall rows and away from the periodic seams (no wrap, no ghost term).
template <bool LAP, bool IN = false>
__device__ __forceinline__ float stencil_T(const float* b, const Geo& g, int x, int y, int axis,
                                           float parity) {
  float s = 0.0f;
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const int c = LAP ? 1 : (axis == 0 ? qcx(i) : qcy(i));
    if (c == 0) continue;
    const float coef = LAP ? 6.0f * qw(i) : 3.0f * qw(i) * c;
    if constexpr (IN) {
      s += coef * b[(y - qcy(i)) * g.nx + x - qcx(i)];
      continue;
    }
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

#define ADJ_NODE                                              \
  const int x = blockIdx.x * kAB + threadIdx.x, y = blockIdx.y; \
  const int n = A.g.nx * A.g.ny;                              \
  const bool live = x < A.g.nx;                               \
  const int k = y * A.g.nx + (live ? x : 0);                  \
  (void)n;
#define TP(pl) (A.tape + (size_t)(pl) * n)
#define AI(pl) (A.ain + (size_t)(kAdjScalar + (pl)) * n)
#define AO(pl) (A.aout + (size_t)(kAdjScalar + (pl)) * n)
// element m of a plane, the offset formed in 32 bits (the host refuses grids
// whose planes would reach 2^31 elements).  The tape and the incoming adjoint
// state are never written by a reverse kernel, and a work plane is read by a
// kernel only where that kernel does not write it (or by the thread that
// writes it, before the write): such reads take the read-only path
// (ld.global.nc), which lets the compiler issue them ahead of the stores of
// earlier directions instead of after them.
#define TPK(pl, m) (__ldg(A.tape + (unsigned)((pl) * n + (m))))
#define AIK(pl, m) (__ldg(A.ain + (unsigned)((kAdjScalar + (pl)) * n + (m))))
#define AOK(pl, m) (A.aout[(unsigned)((kAdjScalar + (pl)) * n + (m))])
#define WKK(pl, m) (A.W[(unsigned)((pl) * n + (m))])
#define WKR(pl, m) (__ldg(A.W + (unsigned)((pl) * n + (m))))
#define SI(m) (__ldg(reinterpret_cast<const float4*>(A.ain) + (m)))
#define SO(m) (reinterpret_cast<float4*>(A.aout)[m])
#define WK(pl) (A.W + (size_t)(pl) * n)

// Full adjoint of pre-collision population i at node m of step t + 1.
// (s: the node's scalar block SB, JX, JY, PHI, read as one 16-byte load)
__device__ __forceinline__ float fb_full(const AdjArgs& A, int n, int i, int m, float4 s) {
  return AIK(AP_F0 + i, m) + s.x + qcx(i) * s.y + qcy(i) * s.z;
}
__device__ __forceinline__ float hb_full(const AdjArgs& A, int n, int i, int m, float4 s) {
  return AIK(AP_H0 + i, m) + s.w;
}

// streaming transpose + collision transpose (+ bounce-back terms); built for
// 7 blocks per SM (72 registers): the kernel is bound by the latency of its
// gathers; measured faster than 8 blocks at 64 registers and than 6 at 80
__global__ void __launch_bounds__(kAB, 7) k_adj_collide(const AdjArgs A) {
  ADJ_NODE
  const Phys& P = A.p;
  const Geo& g = A.g;
  double deta = 0.0;
  if (live) {
    const float phi = TPK(TP_PHI, k), ux = TPK(TP_UX, k), uy = TPK(TP_UY, k);
    const float Fx = TPK(TP_FX, k), Fy = TPK(TP_FY, k), Pr = TPK(TP_PR, k), mu = TPK(TP_MU, k);
    constexpr float c3 = 1.0f / 3.0f;
    const float rho = P.rho_mid + P.drho_half * phi;
    const float irho = 1.0f / rho, rho3 = rho * c3;
    const float mv = P.mu_mid + P.mu_dhalf * phi;
    const float om = 1.0f / (0.5f + 3.0f * mv * irho);
    const float Rx3 = P.drho_half * TPK(TP_GX, k) * c3, Ry3 = P.drho_half * TPK(TP_GY, k) * c3;
    const float uu = ux * ux + uy * uy, uF = ux * Fx + uy * Fy, uR = ux * Rx3 + uy * Ry3;
    const float om1 = 1.0f - om, cff = 1.0f - 0.5f * om, omh1 = 1.0f - P.inv_tau_h;
    float phib = 0.0f, rhob = 0.0f, uxb = 0.0f, uyb = 0.0f, Pb = 0.0f, Fxb = 0.0f, Fyb = 0.0f;
    float Rxb = 0.0f, Ryb = 0.0f, mub = 0.0f, divb = 0.0f, dtxb = 0.0f, dtyb = 0.0f, omb = 0.0f;
    float etab = 0.0f;  // this node's d/d eta (summed over nodes in double)
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      // adjoint of the post-collision population: pull transpose (push), or
      // the reflected population where x + c_i lies beyond a wall
      const int xn = wx(g, x + qcx(i));
      int yn = y + qcy(i);
      float fpb, hpb;
      if (g.wall && (yn < 0 || yn >= g.ny)) {
        const int o = qopp(i);
        const float4 sk = SI(k);
        fpb = fb_full(A, n, o, k, sk);
        hpb = hb_full(A, n, o, k, sk);
        const float cu = qcx(i) * (yn < 0 ? P.uwb : P.uwt);
        rhob += -2.0f * qw(i) * cu * fpb;
        phib += -6.0f * qw(i) * cu * hpb;
      } else {
        if (!g.wall) yn = yn < 0 ? yn + g.ny : (yn >= g.ny ? yn - g.ny : yn);
        const int m = yn * g.nx + xn;
        const float4 sm = SI(m);
        fpb = fb_full(A, n, i, m, sm);
        hpb = hb_full(A, n, i, m, sm);
      }
      const float cu = qcx(i) * ux + qcy(i) * uy;
      const float s = 3.0f * cu + 4.5f * cu * cu - 1.5f * uu;
      const float feq = qw(i) * (Pr + rho3 * s);
      const float cF = qcx(i) * Fx + qcy(i) * Fy;
      const float cR = qcx(i) * Rx3 + qcy(i) * Ry3;
      const float Fi = qw(i) * ((1.0f + s) * (cF - uF) + s * (cR - uR));
      AOK(AP_F0 + i, k) = om1 * fpb;
      omb += fpb * (-TPK(TP_F0 + i, k) + feq - 0.5f * Fi);
      const float feqb = om * fpb, Fib = cff * fpb;
      Pb += qw(i) * feqb;
      rhob += (qw(i) * c3) * s * feqb;
      float sb = qw(i) * rho3 * feqb;
      sb += qw(i) * ((cF - uF) + (cR - uR)) * Fib;
      const float k1 = qw(i) * (1.0f + s) * Fib, k2 = qw(i) * s * Fib;
      Fxb += k1 * (qcx(i) - ux);
      Fyb += k1 * (qcy(i) - uy);
      uxb += -k1 * Fx - k2 * Rx3;
      uyb += -k1 * Fy - k2 * Ry3;
      Rxb += k2 * (qcx(i) - ux);  // times 1/3 below
      Ryb += k2 * (qcy(i) - uy);
      uxb += sb * ((3.0f + 9.0f * cu) * qcx(i) - 3.0f * ux);
      uyb += sb * ((3.0f + 9.0f * cu) * qcy(i) - 3.0f * uy);
      // h
      AOK(AP_H0 + i, k) = omh1 * hpb;
      const float heqb = hpb * P.inv_tau_h, Hb = P.hforce * hpb;
      if (i == 0) {
        phib += heqb;
        mub += (qw(0) - 1.0f) * P.eta * heqb;
        etab += (qw(0) - 1.0f) * mu * heqb;
      } else {
        mub += qw(i) * P.eta * heqb;
        etab += qw(i) * mu * heqb;
        phib += 3.0f * qw(i) * cu * heqb;
        uxb += 3.0f * qw(i) * phi * qcx(i) * heqb;
        uyb += 3.0f * qw(i) * phi * qcy(i) * heqb;
      }
      divb += (i == 0 ? qw(0) - 1.0f : qw(i)) * P.acoef * Hb;
      dtxb += 3.0f * qw(i) * qcx(i) * Hb;
      dtyb += 3.0f * qw(i) * qcy(i) * Hb;
    }
    // omega = 1/tau_f, tau_f = 1/2 + 3 mu_v / rho
    const float taub = -om * om * omb;
    phib += P.mu_dhalf * (3.0f * irho * taub);
    rhob += -3.0f * mv * (irho * irho) * taub;
    Rxb *= c3;
    Ryb *= c3;
    deta = (double)etab;
    WKK(B_PHI, k) = phib;
    WKK(B_RHO, k) = rhob;
    WKK(B_UX, k) = uxb;
    WKK(B_UY, k) = uyb;
    WKK(B_P, k) = Pb;
    WKK(B_FX, k) = Fxb;
    WKK(B_FY, k) = Fyb;
    WKK(B_GX, k) = P.drho_half * Rxb;  // R = (rho1 - rho2)/2 grad phi
    WKK(B_GY, k) = P.drho_half * Ryb;
    WKK(B_MU, k) = mub;
    WKK(B_DIV, k) = divb;
    WKK(B_DTX, k) = dtxb;
    WKK(B_DTY, k) = dtyb;
  }
  acc_add(A.acc, 0.0, 0.0, deta, 0.0);
}

// Values of the middle and late stages at one node.
struct Tail {
  float phib, Gxb, Gyb, mub, Lb, w0, w1, w2;
};

// div(phi u) and d_t(phi u) = p - q, the incoming adjoint of (phi u)^t, then
// p = phi u, P = S + u.R/6, u = (3 j + F/2)/rho, F = F_sf + (rho - rho0) g,
// rho(phi), and the pointwise part of the force of the form; leaves in
// w0..w2 what the force's stencil transposes read.  The node's outputs to the
// adjoint state (q and the scalar block) are written when `own`.
template <bool IN = false>
__device__ __forceinline__ Tail mid_node(const AdjArgs& A, int n, int x, int y, int k, bool own,
                                         double& dk, double& ds) {
  const Phys& P = A.p;
  const Geo& g = A.g;
  const float* divb = WK(B_DIV);
  // p_x is read as parity -1 with an additive 2 u_w phi at the wall ghosts,
  // p_y with parity -1; periodic wraps
  float pxb = stencil_T<false, IN>(divb, g, x, y, 0, -1.0f);
  float pyb = stencil_T<false, IN>(divb, g, x, y, 1, -1.0f);
  Tail o;
  o.phib = WKR(B_PHI, k);
  if (!IN && g.wall && (y == 0 || y == g.ny - 1)) {
    // ghost adjoint of p_x at (x, -1) or (x, ny): nodes of this row whose
    // stencil reads it; its 2 u_w phi(x, row) part goes to phi
    const int cyw = y == 0 ? -1 : 1;
    float ga = 0.0f;
#pragma unroll
    for (int i = 1; i < 9; ++i)
      if (qcy(i) == cyw) ga += 3.0f * qw(i) * qcx(i) * divb[y * g.nx + wx(g, x - qcx(i))];
    o.phib += 2.0f * (y == 0 ? P.uwb : P.uwt) * ga;
  }
  pxb += AIK(AP_QX, k);
  pyb += AIK(AP_QY, k);
  const float dtxb = A.first ? 0.0f : WKR(B_DTX, k), dtyb = A.first ? 0.0f : WKR(B_DTY, k);
  pxb += dtxb;
  pyb += dtyb;
  // macroscopic relations
  const float phi = TPK(TP_PHI, k), ux = TPK(TP_UX, k), uy = TPK(TP_UY, k);
  const float gx = TPK(TP_GX, k), gy = TPK(TP_GY, k);
  constexpr float c6 = 1.0f / 6.0f;
  const float rho = P.rho_mid + P.drho_half * phi;
  const float irho = 1.0f / rho;
  const float Rx = P.drho_half * gx, Ry = P.drho_half * gy;
  const float Pb = WKR(B_P, k);
  o.phib += pxb * ux + pyb * uy;
  const float uxb = WKR(B_UX, k) + phi * pxb + Rx * c6 * Pb;
  const float uyb = WKR(B_UY, k) + phi * pyb + Ry * c6 * Pb;
  o.Gxb = WKR(B_GX, k) + P.drho_half * (ux * c6 * Pb);
  o.Gyb = WKR(B_GY, k) + P.drho_half * (uy * c6 * Pb);
  if (own) {
    AOK(AP_QX, k) = -dtxb;
    AOK(AP_QY, k) = -dtyb;
    // (PHI, the w component, is written by the finishing stage)
    SO(k) = make_float4(Pb, 3.0f * uxb * irho, 3.0f * uyb * irho, 0.0f);
  }
  const float Fxb = WKR(B_FX, k) + 0.5f * uxb * irho;  // adjoint of F_sf
  const float Fyb = WKR(B_FY, k) + 0.5f * uyb * irho;
  float rhob = WKR(B_RHO, k) - (ux * uxb + uy * uyb) * irho;
  rhob += P.gx * Fxb + P.gy * Fyb;
  o.phib += P.drho_half * rhob;
  // pointwise part of the force
  o.mub = WKR(B_MU, k);
  o.Lb = o.w0 = o.w1 = o.w2 = 0.0f;
  const float a0 = TPK(TP_A0, k), a1 = TPK(TP_A1, k);
  switch (A.form) {
    case kSTF1:
    case kSTF2:  // F_sf = kappa (a0, a1) / kappa: the tape holds F_sf
      dk += (double)((Fxb * a0 + Fyb * a1) * (1.0f / P.kappa));
      o.w0 = Fxb;
      o.w1 = Fyb;
      break;
    case kCPF1:  // F = -phi grad mu, tape: grad mu
      o.phib += -(a0 * Fxb + a1 * Fyb);
      o.w0 = -phi * Fxb;
      o.w1 = -phi * Fyb;
      break;
    case kCPF2: {
      const float mu = TPK(TP_MU, k);
      o.mub += gx * Fxb + gy * Fyb;
      o.Gxb += mu * Fxb;
      o.Gyb += mu * Fyb;
      break;
    }
    case kPF1: {
      const float L = TPK(TP_L, k);
      o.Gxb += -P.kappa * L * Fxb;
      o.Gyb += -P.kappa * L * Fyb;
      o.Lb = -P.kappa * (gx * Fxb + gy * Fyb);
      dk += (double)(-(gx * Fxb + gy * Fyb) * L);
      break;
    }
    case kPF2:  // F = kappa phi grad lap phi, tape: grad lap phi
      o.phib += P.kappa * (a0 * Fxb + a1 * Fyb);
      dk += (double)(phi * (a0 * Fxb + a1 * Fyb));
      o.w0 = P.kappa * phi * Fxb;
      o.w1 = P.kappa * phi * Fyb;
      break;
    default: {  // CSF, tape: div n
      const float divn = a0;
      const float a = sqrtf(gx * gx + gy * gy);
      const float GF = gx * Fxb + gy * Fyb;
      if (A.form == kCSF1) {
        o.Gxb += -P.kappa * a * divn * Fxb;
        o.Gyb += -P.kappa * a * divn * Fyb;
        const float ab = -P.kappa * divn * GF;
        o.w2 = -P.kappa * a * GF;
        dk += (double)(-GF * a * divn);
        if (a > 0.0f) {
          const float ia = 1.0f / a;
          o.Gxb += ab * gx * ia;
          o.Gyb += ab * gy * ia;
        }
      } else {
        o.Gxb += -P.half_sigma * divn * Fxb;
        o.Gyb += -P.half_sigma * divn * Fyb;
        o.w2 = -P.half_sigma * GF;
        ds += (double)(-0.5f * GF * divn);
      }
    }
  }
  return o;
}

// Stencil part of the force adjoint, then mu = 4 beta phi (phi^2 - 1) - kappa
// lap phi, at node k with its middle-stage values v; st(field, axis, parity)
// is the transposed first-derivative stencil of w0, w1 or w2 (field 0, 1, 2).
template <class ST>
__device__ __forceinline__ void late_node(const AdjArgs& A, int n, int k, Tail& v, const ST& st,
                                          double& db, double& dk) {
  const Phys& P = A.p;
  const float gx = TPK(TP_GX, k), gy = TPK(TP_GY, k), phi = TPK(TP_PHI, k);
  switch (A.form) {
    case kSTF1:
    case kSTF2: {
      float txx = -P.kappa * st(0, 0, 1.0f);
      const float txy = -P.kappa * (st(0, 1, -1.0f) + st(1, 0, -1.0f));
      float tyy = -P.kappa * st(1, 1, 1.0f);
      if (A.form == kSTF2) {
        const float g2b = P.kappa * (st(0, 0, 1.0f) + st(1, 1, 1.0f));
        txx += g2b;
        tyy += g2b;
      }
      v.Gxb += 2.0f * gx * txx + gy * txy;
      v.Gyb += gx * txy + 2.0f * gy * tyy;
      break;
    }
    case kCPF1:
      v.mub += st(0, 0, 1.0f) + st(1, 1, 1.0f);
      break;
    case kPF2:
      v.Lb += st(0, 0, 1.0f) + st(1, 1, 1.0f);
      break;
    case kCSF1:
    case kCSF2: {
      const float nxb = st(2, 0, 1.0f);
      const float nyb = st(2, 1, -1.0f);
      const float ir = rsqrtf(gx * gx + gy * gy + P.eps2);
      const float gn = gx * nxb + gy * nyb, ir3 = ir * ir * ir;
      v.Gxb += nxb * ir - gx * gn * ir3;
      v.Gyb += nyb * ir - gy * gn * ir3;
      break;
    }
    default:
      break;
  }
  v.phib += P.beta4 * (3.0f * phi * phi - 1.0f) * v.mub;
  v.Lb += -P.kappa * v.mub;
  db += (double)(phi * (phi * phi - 1.0f) * v.mub);
  dk += (double)(-TPK(TP_L, k) * v.mub);
}

// Transposed stencils on a shared-memory tile of row stride S: node at local
// index c, domain row y (the wall rule of stencil_T, periodic seams already
// resolved by the tile's layout).
template <bool LAP, int S, bool IN = false>
__device__ __forceinline__ float stencil_T_tile(const float* b, int c, int y, const Geo& g,
                                                int axis, float parity) {
  float s = 0.0f;
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const int cxi = qcx(i), cyi = qcy(i);
    const int cc = LAP ? 1 : (axis == 0 ? cxi : cyi);
    if (cc == 0) continue;
    const float coef = LAP ? 6.0f * qw(i) : 3.0f * qw(i) * cc;
    if (!IN && g.wall) {
      const int ys = y - cyi;
      if (ys >= 0 && ys < g.ny) s += coef * b[c - cxi - cyi * S];
      if ((y == 0 && cyi == -1) || (y == g.ny - 1 && cyi == 1)) s += parity * coef * b[c - cxi];
    } else {
      s += coef * b[c - cxi - cyi * S];
    }
  }
  if (LAP) s -= (10.0f / 3.0f) * b[c];
  return s;
}

// The three stages after the collision transpose, fused over a 32 x 8 tile:
// the middle stage on the tile + 2 ring, the late stage on the tile + 1 ring
// (its stencils read the middle stage's w0..w2 in shared memory), the
// finishing transposes of grad phi and lap phi on the tile.  A ring node
// outside the domain beyond a wall is skipped (no stencil reads it); every
// parameter gradient term comes from the tile's own nodes.  IN: the tile + 3
// ring lies inside the domain, off the wall rows and the periodic seams (no
// wrap, no ghost terms).
constexpr int kTW = 32, kTH = 8, kTS = kTW + 4, kTN = kTS * (kTH + 4);
// 256 threads, four CTAs per SM (64 registers; the 512 tiles of a 512 x 256
// grid still fit one wave): measured faster than six CTAs per SM at 40
// registers, than the same with the stage loops unrolled, and than one
// thread per ring node (448 threads, three or four CTAs per SM)
constexpr int kTailThreads = 256, kTailBlocks = 4;
template <bool IN>
__device__ __forceinline__ void tail_tile(const AdjArgs& A, float (*sw)[kTN], float (*sv)[kTN],
                                          int x0, int y0, double& db, double& dk, double& ds) {
  const int n = A.g.nx * A.g.ny;
  const Geo& g = A.g;
  // node (lx, ly) of the tile + 2 ring: domain coordinates, or false beyond a wall
  auto node = [&](int lx, int ly, int& x, int& y) {
    if constexpr (IN) {
      x = x0 - 2 + lx;
      y = y0 - 2 + ly;
      return true;
    }
    x = wx(g, x0 - 2 + lx);
    y = y0 - 2 + ly;
    if (g.wall) return y >= 0 && y < g.ny;
    y = y < 0 ? y + g.ny : (y >= g.ny ? y - g.ny : y);
    return true;
  };
  auto owned = [&](int lx, int ly) {
    return lx >= 2 && lx < kTW + 2 && ly >= 2 && ly < kTH + 2 &&
           (IN || (x0 + lx - 2 < g.nx && y0 + ly - 2 < g.ny));
  };
  for (int c = threadIdx.x; c < kTN; c += kTailThreads) {
    const int ly = c / kTS, lx = c - ly * kTS;
    int x, y;
    if (!node(lx, ly, x, y)) continue;
    const bool own = owned(lx, ly);
    double dkn = 0.0, dsn = 0.0;
    const Tail t = mid_node<IN>(A, n, x, y, y * g.nx + x, own, dkn, dsn);
    if (own) {
      dk += dkn;
      ds += dsn;
    }
    sw[0][c] = t.w0;
    sw[1][c] = t.w1;
    sw[2][c] = t.w2;
    sv[0][c] = t.phib;
    sv[1][c] = t.Gxb;
    sv[2][c] = t.Gyb;
    sv[3][c] = t.mub;
    sv[4][c] = t.Lb;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < kTN; c += kTailThreads) {
    const int ly = c / kTS, lx = c - ly * kTS;
    if (lx < 1 || lx > kTW + 2 || ly < 1 || ly > kTH + 2) continue;  // tile + 1 ring
    int x, y;
    if (!node(lx, ly, x, y)) continue;
    Tail v;
    v.phib = sv[0][c];
    v.Gxb = sv[1][c];
    v.Gyb = sv[2][c];
    v.mub = sv[3][c];
    v.Lb = sv[4][c];
    const auto st = [&](int f, int axis, float parity) {
      return stencil_T_tile<false, kTS, IN>(sw[f], c, y, g, axis, parity);
    };
    double dbn = 0.0, dkn = 0.0;
    late_node(A, n, y * g.nx + x, v, st, dbn, dkn);
    if (owned(lx, ly)) {
      db += dbn;
      dk += dkn;
    }
    sv[0][c] = v.phib;  // the late stage reads only w0..w2 of other nodes
    sv[1][c] = v.Gxb;
    sv[2][c] = v.Gyb;
    sv[4][c] = v.Lb;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < kTN; c += kTailThreads) {
    const int ly = c / kTS, lx = c - ly * kTS;
    if (!owned(lx, ly)) continue;
    int x, y;
    node(lx, ly, x, y);
    const int k = y * g.nx + x;
    reinterpret_cast<float*>(A.aout)[4 * k + 3] =  // the PHI (w) component of SO(k)
        sv[0][c] + stencil_T_tile<false, kTS, IN>(sv[1], c, y, g, 0, 1.0f) +
        stencil_T_tile<false, kTS, IN>(sv[2], c, y, g, 1, 1.0f) +
        stencil_T_tile<true, kTS, IN>(sv[4], c, y, g, 0, 1.0f);
  }
}

__global__ void __launch_bounds__(kTailThreads, kTailBlocks) k_adj_tail(const AdjArgs A) {
  const Geo& g = A.g;
  __shared__ float sw[3][kTN];   // w0, w1, w2
  __shared__ float sv[5][kTN];   // phib, Gxb, Gyb, mub, Lb
  const int x0 = blockIdx.x * kTW, y0 = blockIdx.y * kTH;
  double dk = 0.0, ds = 0.0, db = 0.0;
  // the middle stage's divergence transpose reads the tile + 3 ring
  const bool in = x0 >= 3 && x0 + kTW + 3 <= g.nx && y0 >= 3 && y0 + kTH + 3 <= g.ny;
  if (in) tail_tile<true>(A, sw, sv, x0, y0, db, dk, ds);
  else tail_tile<false>(A, sw, sv, x0, y0, db, dk, ds);
  // one FP64 block reduction of the four accumulators
  constexpr int kWarps = kTailThreads / 32;
  __shared__ double red[kWarps][4];
  double v4[4] = {db, dk, 0.0, ds};
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v4[q] += __shfl_down_sync(0xffffffffu, v4[q], o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < 4; ++q) red[w][q] = v4[q];
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int j = 0; j < kWarps; ++j) s += red[j][threadIdx.x];
    if (s != 0.0) atomicAdd(&A.acc[threadIdx.x], s);
  }
}

// Reverse of one step: adjoint state at t + 1 (A.ain) -> at t (A.aout), with
// the tape of step t.
// The stages after the collision transpose run as one tiled kernel on every
// grid (measured on the drop in shear against three one-thread-per-node
// kernels exchanging their values through work planes: 4.5x against 4.6x the
// forward at 131 072 nodes, 6.5x against 6.8x at 524 288, 6.2x against 6.3x
// at 2 097 152).
cudaError_t launch_adjoint_step(const AdjArgs& A, cudaStream_t s) {
  const dim3 grid((A.g.nx + kAB - 1) / kAB, A.g.ny);
  k_adj_collide<<<grid, kAB, 0, s>>>(A);
  const dim3 tiles((A.g.nx + kTW - 1) / kTW, (A.g.ny + kTH - 1) / kTH);
  k_adj_tail<<<tiles, kTailThreads, 0, s>>>(A);
  return cudaGetLastError();
}

// ---- initial state: h = h^eq(phi0, mu0, 0), f = 0 ------------------------------
__global__ void __launch_bounds__(kAB) k_adj_init_pt(const AdjArgs A, const float* phi0) {
  ADJ_NODE
  double db = 0.0, dk = 0.0, de = 0.0;
  if (live) {
    const Phys& P = A.p;
    const float phi = phi0[k];
    const float L = lapfw(phi0, A.g, x, y);
    const float mu = P.beta4 * phi * ((phi - 1.0f) * (phi + 1.0f)) - P.kappa * L;
    const float4 sk = SI(k);
    const float hb0 = hb_full(A, n, 0, k, sk);
    float hsum = (qw(0) - 1.0f) * hb0;
#pragma unroll
    for (int i = 1; i < 9; ++i) hsum += qw(i) * hb_full(A, n, i, k, sk);
    const float mub = P.eta * hsum;
    de = (double)(mu * hsum);
    db = (double)(phi * (phi * phi - 1.0f) * mub);
    dk = (double)(-L * mub);
    WKK(B_PHI, k) = hb0 + P.beta4 * (3.0f * phi * phi - 1.0f) * mub;
    WKK(B_L, k) = -P.kappa * mub;
  }
  acc_add(A.acc, db, dk, de, 0.0);
}

__global__ void __launch_bounds__(kAB) k_adj_init_out(const AdjArgs A, float* dphi0) {
  ADJ_NODE
  if (!live) return;
  dphi0[k] = WKK(B_PHI, k) + stencil_T<true>(WK(B_L), A.g, x, y, 0, 1.0f);
}

cudaError_t launch_adjoint_init(const AdjArgs& A, const float* phi0, float* dphi0,
                                cudaStream_t s) {
  const dim3 grid((A.g.nx + kAB - 1) / kAB, A.g.ny);
  k_adj_init_pt<<<grid, kAB, 0, s>>>(A, phi0);
  k_adj_init_out<<<grid, kAB, 0, s>>>(A, dphi0);
  return cudaGetLastError();
}

// ---- taping step ----------------------------------------------------------------
template <int FORM>
cudaError_t tape_form(const StepArgs* a, cudaStream_t s) {
  constexpr int kBytes = Fields<FORM, true>::BYTES;
  if (!a)  // set-up: the shared-memory attribute (before any stream capture)
    return cudaFuncSetAttribute(k_step_tape<FORM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kBytes);
  const int ntiles = ((a->L.nx + kTX - 1) / kTX) * ((a->L.ny + kTY - 1) / kTY);
  k_step_tape<FORM><<<ntiles, kThreadsGather, kBytes, s>>>(*a);
  return cudaGetLastError();
}

cudaError_t tape_dispatch(int form, const StepArgs* a, cudaStream_t s) {
  switch (form) {
    case kSTF1: return tape_form<kSTF1>(a, s);
    case kSTF2: return tape_form<kSTF2>(a, s);
    case kCPF1: return tape_form<kCPF1>(a, s);
    case kCPF2: return tape_form<kCPF2>(a, s);
    case kPF1: return tape_form<kPF1>(a, s);
    case kPF2: return tape_form<kPF2>(a, s);
    case kCSF1: return tape_form<kCSF1>(a, s);
    case kCSF2: return tape_form<kCSF2>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t setup_tape_step(int form) { return tape_dispatch(form, nullptr, nullptr); }

cudaError_t launch_tape_step(int form, const StepArgs& a, cudaStream_t s) {
  return tape_dispatch(form, &a, s);
}

}  // namespace pflbm

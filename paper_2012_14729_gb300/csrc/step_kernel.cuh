// Fused coupled step of the phase-field lattice Boltzmann method (Sec. 3 of
// Zhang, Liang & Guo, arXiv 2012.14729) for sm_103a.
//
// One CTA owns a kTX x kTY tile of nodes and runs the whole time step for it
// in four passes over shared memory, recomputing what its neighbours need on
// a halo instead of exchanging it through HBM:
//   pass 1  phi = sum_i h_i on the tile + 3 ring (pull of h, Eq. mac)
//   pass 2  grad phi, lap phi (Eqs. ICS-1st, ICS-sec), mu (Eq.
//           chemical_potential) and the form's level-1 fields on tile + 2
//   pass 3  interfacial + gravity force (Sec. 2.2), rho, u and phi u on
//           tile + 1 (pull of f, Eq. mac)
//   pass 4  on the tile: P, div(phi u), d_t(phi u), BGK collision of f and h
//           with F_i and H_i (Eqs. fh, P_LBM, CH_LB_force), store of the
//           post-collision populations; streaming is the next step's pull.
// HBM traffic per node and step is the algorithmic state: 18 populations read
// and written plus (phi u) read and written; halo re-reads hit L1/L2.
//
// Walls (Sec. 4, half-way bounce-back): populations are stored with one
// ghost row below and above the domain.  A node next to a wall writes the
// bounced populations (with the moving-wall term) into the ghost row, where
// the next step's pull finds them.  Scalar stencils see mirror ghosts (row
// -k equals row k-1), and the ghost of phi u is phi (2 u_w - u) of the
// mirrored node.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"

namespace pflbm {

// ---------------------------------------------------------------------------
// D2Q9 lattice: c_0..c_8 = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),
// (-1,-1),(1,-1), weights 4/9, 1/9, 1/36 (Sec. 3)
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int qcx(int i) {
  return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int qcy(int i) {
  return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr float qw(int i) {
  return i == 0 ? 4.0f / 9.0f : (i < 5 ? 1.0f / 9.0f : 1.0f / 36.0f);
}
__host__ __device__ constexpr int qopp(int i) {
  return i == 0 ? 0 : (i < 5 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
}

enum Form { kSTF1 = 0, kSTF2, kCPF1, kCPF2, kPF1, kPF2, kCSF1, kCSF2 };

// Number of form-specific level-1 fields kept in shared memory.
template <int FORM>
__host__ __device__ constexpr int extra_fields() {
  return (FORM == kSTF1 || FORM == kSTF2) ? 3 : ((FORM == kCSF1 || FORM == kCSF2) ? 2 : 0);
}

// ---------------------------------------------------------------------------
// storage formats
// ---------------------------------------------------------------------------
struct StoreF32 {
  static constexpr bool kSplitH0 = false;
  using T = float;
  __device__ static __forceinline__ float dec(T v, float w_inv_scale) { return v; }
  __device__ static __forceinline__ T enc(float v, float scale_over_w) { return v; }
};
struct StoreF16 {
  static constexpr bool kSplitH0 = true;
  using T = __half;
  __device__ static __forceinline__ float dec(T v, float w_inv_scale) {
    return __half2float(v) * w_inv_scale;
  }
  __device__ static __forceinline__ T enc(float v, float scale_over_w) {
    return __float2half_rn(v * scale_over_w);
  }
};
struct StoreBF16 {
  static constexpr bool kSplitH0 = true;
  using T = __nv_bfloat16;
  __device__ static __forceinline__ float dec(T v, float w_inv_scale) {
    return __bfloat162float(v) * w_inv_scale;
  }
  __device__ static __forceinline__ T enc(float v, float scale_over_w) {
    return __float2bfloat16_rn(v * scale_over_w);
  }
};

// f_i, population i at storage index idx
template <class ST, int I>
__device__ __forceinline__ float load_f(const StepArgs& a, int idx) {
  using T = typename ST::T;
  const T* base = reinterpret_cast<const T*>(a.f_in) + (size_t)I * a.L.plane;
  if constexpr (ST::kSplitH0) return ST::dec(__ldg(base + idx), qw(I) * a.p.inv_sf);
  else return __ldg(base + idx);
}
template <class ST, int I>
__device__ __forceinline__ float load_h(const StepArgs& a, int idx) {
  using T = typename ST::T;
  if constexpr (ST::kSplitH0) {
    if constexpr (I == 0) return __ldg(a.h0_in + idx);
    else {
      const T* base = reinterpret_cast<const T*>(a.h_in) + (size_t)(I - 1) * a.L.plane;
      return ST::dec(__ldg(base + idx), qw(I) * a.p.inv_sh);
    }
  } else {
    const T* base = reinterpret_cast<const T*>(a.h_in) + (size_t)I * a.L.plane;
    return __ldg(base + idx);
  }
}
template <class ST, int I>
__device__ __forceinline__ void store_f(const StepArgs& a, int idx, float v) {
  using T = typename ST::T;
  T* base = reinterpret_cast<T*>(a.f_out) + (size_t)I * a.L.plane;
  if constexpr (ST::kSplitH0) base[idx] = ST::enc(v, a.p.sf * (1.0f / qw(I)));
  else base[idx] = v;
}
template <class ST, int I>
__device__ __forceinline__ void store_h(const StepArgs& a, int idx, float v) {
  using T = typename ST::T;
  if constexpr (ST::kSplitH0) {
    if constexpr (I == 0) a.h0_out[idx] = v;
    else {
      T* base = reinterpret_cast<T*>(a.h_out) + (size_t)(I - 1) * a.L.plane;
      base[idx] = ST::enc(v, a.p.sh * (1.0f / qw(I)));
    }
  } else {
    T* base = reinterpret_cast<T*>(a.h_out) + (size_t)I * a.L.plane;
    base[idx] = v;
  }
}

// ---------------------------------------------------------------------------
// index helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int wrap(int v, int n) {
  if (v >= 0 && v < n) return v;
  v %= n;
  return v < 0 ? v + n : v;
}
// Row of a scalar-field node: periodic wrap, or mirror about the walls.
__device__ __forceinline__ int map_row(int y, int ny, int wall) {
  if (y >= 0 && y < ny) return y;
  if (!wall) return wrap(y, ny);
  while (y < 0 || y >= ny) y = (y < 0) ? -y - 1 : 2 * ny - 1 - y;
  return y;
}

// Storage indices of the 9 pulled populations of node (x, y), 0 <= x < nx,
// 0 <= y < ny: population i comes from (x - cx_i, y - cy_i); storage row is
// domain row + 1 (ghost rows 0 and ny + 1 hold bounced populations).
struct Pull {
  int i[9];
};
__device__ __forceinline__ Pull pull_idx(const Lattice& L, int x, int y) {
  int xm = x + 1, xp = x - 1;  // source columns for cx = -1 and cx = +1
  if (xm >= L.nx) xm -= L.nx;
  if (xp < 0) xp += L.nx;
  int ym = y + 1, yp = y - 1;  // source rows for cy = -1 and cy = +1
  if (!L.wall) {
    if (ym >= L.ny) ym -= L.ny;
    if (yp < 0) yp += L.ny;
  }
  const int r0 = (y + 1) * L.nx, rm = (ym + 1) * L.nx, rp = (yp + 1) * L.nx;
  Pull p;
  p.i[0] = r0 + x;
  p.i[1] = r0 + xp;
  p.i[2] = rp + x;
  p.i[3] = r0 + xm;
  p.i[4] = rm + x;
  p.i[5] = rp + xp;
  p.i[6] = rp + xm;
  p.i[7] = rm + xm;
  p.i[8] = rm + xp;
  return p;
}

template <class ST>
__device__ __forceinline__ float pull_phi(const StepArgs& a, const Pull& q) {
  // summed in direction order 0..8
  float s = load_h<ST, 0>(a, q.i[0]);
  s += load_h<ST, 1>(a, q.i[1]);
  s += load_h<ST, 2>(a, q.i[2]);
  s += load_h<ST, 3>(a, q.i[3]);
  s += load_h<ST, 4>(a, q.i[4]);
  s += load_h<ST, 5>(a, q.i[5]);
  s += load_h<ST, 6>(a, q.i[6]);
  s += load_h<ST, 7>(a, q.i[7]);
  s += load_h<ST, 8>(a, q.i[8]);
  return s;
}

template <class ST>
__device__ __forceinline__ void pull_f(const StepArgs& a, const Pull& q, float* f) {
  f[0] = load_f<ST, 0>(a, q.i[0]);
  f[1] = load_f<ST, 1>(a, q.i[1]);
  f[2] = load_f<ST, 2>(a, q.i[2]);
  f[3] = load_f<ST, 3>(a, q.i[3]);
  f[4] = load_f<ST, 4>(a, q.i[4]);
  f[5] = load_f<ST, 5>(a, q.i[5]);
  f[6] = load_f<ST, 6>(a, q.i[6]);
  f[7] = load_f<ST, 7>(a, q.i[7]);
  f[8] = load_f<ST, 8>(a, q.i[8]);
}
template <class ST>
__device__ __forceinline__ void pull_h(const StepArgs& a, const Pull& q, float* h) {
  h[0] = load_h<ST, 0>(a, q.i[0]);
  h[1] = load_h<ST, 1>(a, q.i[1]);
  h[2] = load_h<ST, 2>(a, q.i[2]);
  h[3] = load_h<ST, 3>(a, q.i[3]);
  h[4] = load_h<ST, 4>(a, q.i[4]);
  h[5] = load_h<ST, 5>(a, q.i[5]);
  h[6] = load_h<ST, 6>(a, q.i[6]);
  h[7] = load_h<ST, 7>(a, q.i[7]);
  h[8] = load_h<ST, 8>(a, q.i[8]);
}

// Central-scheme derivatives (Eq. ICS-1st) of a shared-memory field at
// element c with row stride S: d/dx = 3 sum_i w_i c_ix a(x + c_i).
template <int S>
__device__ __forceinline__ float ics_dx(const float* a, int c) {
  return (a[c + 1] - a[c - 1]) * (1.0f / 3.0f) +
         ((a[c + S + 1] - a[c + S - 1]) + (a[c - S + 1] - a[c - S - 1])) * (1.0f / 12.0f);
}
template <int S>
__device__ __forceinline__ float ics_dy(const float* a, int c) {
  return (a[c + S] - a[c - S]) * (1.0f / 3.0f) +
         ((a[c + S + 1] - a[c - S + 1]) + (a[c + S - 1] - a[c - S - 1])) * (1.0f / 12.0f);
}

// ---------------------------------------------------------------------------
// the fused step kernel
// ---------------------------------------------------------------------------
template <int FORM, class ST>
__global__ void __launch_bounds__(kThreads) k_step(const StepArgs a) {
  constexpr int B3X = kTX + 6, B3Y = kTY + 6;
  constexpr int B2X = kTX + 4, B2Y = kTY + 4;
  constexpr int B1X = kTX + 2, B1Y = kTY + 2;
  constexpr int N2 = B2X * B2Y, N1 = B1X * B1Y;
  constexpr int NE = extra_fields<FORM>();
  // level-1 field slots in s2
  constexpr int GX = 0, GY = 1, LAP = 2, MU = 3, E0 = 4;
  // ring-1 slots in s1
  constexpr int FX = 0, FY = 1, UX = 2, UY = 3, PUX = 4, PUY = 5;

  __shared__ float sPhi[B3X * B3Y];
  __shared__ float s2[(4 + NE) * N2];
  __shared__ float s1[6 * N1];

  const Lattice L = a.L;
  const Phys& P = a.p;
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
  const int tid = threadIdx.x;

  // ---- pass 1: phi on tile + 3 ------------------------------------------------
  for (int k = tid; k < B3X * B3Y; k += kThreads) {
    const int ly = k / B3X, lx = k - ly * B3X;
    const int gx = wrap(x0 - 3 + lx, L.nx);
    const int gy = map_row(y0 - 3 + ly, L.ny, L.wall);
    sPhi[k] = pull_phi<ST>(a, pull_idx(L, gx, gy));
  }
  __syncthreads();

  // ---- pass 2: grad phi, lap phi, mu, level-1 fields on tile + 2 -------------
  for (int k = tid; k < N2; k += kThreads) {
    const int ly = k / B2X, lx = k - ly * B2X;
    const int c = (ly + 1) * B3X + lx + 1;
    const float pc = sPhi[c];
    const float gx = ics_dx<B3X>(sPhi, c);
    const float gy = ics_dy<B3X>(sPhi, c);
    // Eq. ICS-sec: (2/cs^2) sum w_i (phi_i - phi_c)
    const float lap = ((sPhi[c + 1] - pc) + (sPhi[c - 1] - pc) + (sPhi[c + B3X] - pc) +
                       (sPhi[c - B3X] - pc)) * (2.0f / 3.0f) +
                      ((sPhi[c + B3X + 1] - pc) + (sPhi[c + B3X - 1] - pc) +
                       (sPhi[c - B3X + 1] - pc) + (sPhi[c - B3X - 1] - pc)) * (1.0f / 6.0f);
    s2[GX * N2 + k] = gx;
    s2[GY * N2 + k] = gy;
    s2[LAP * N2 + k] = lap;
    s2[MU * N2 + k] = P.beta4 * pc * ((pc - 1.0f) * (pc + 1.0f)) - P.kappa * lap;
    if constexpr (FORM == kSTF1 || FORM == kSTF2) {
      s2[(E0 + 0) * N2 + k] = gx * gx;
      s2[(E0 + 1) * N2 + k] = gx * gy;
      s2[(E0 + 2) * N2 + k] = gy * gy;
    }
    if constexpr (FORM == kCSF1 || FORM == kCSF2) {
      const float inv = rsqrtf(gx * gx + gy * gy + P.eps2);
      s2[(E0 + 0) * N2 + k] = gx * inv;
      s2[(E0 + 1) * N2 + k] = gy * inv;
    }
  }
  __syncthreads();

  // ---- pass 3: force, rho, u, phi u on tile + 1 -----------------------------
  for (int k = tid; k < N1; k += kThreads) {
    const int ly = k / B1X, lx = k - ly * B1X;
    const int c2 = (ly + 1) * B2X + lx + 1;
    const float phi = sPhi[(ly + 2) * B3X + lx + 2];
    const float gx = s2[GX * N2 + c2], gy = s2[GY * N2 + c2];
    float Fx, Fy;
    if constexpr (FORM == kSTF1 || FORM == kSTF2) {
      const float* txx = s2 + (E0 + 0) * N2;
      const float* txy = s2 + (E0 + 1) * N2;
      const float* tyy = s2 + (E0 + 2) * N2;
      Fx = -P.kappa * (ics_dx<B2X>(txx, c2) + ics_dy<B2X>(txy, c2));
      Fy = -P.kappa * (ics_dx<B2X>(txy, c2) + ics_dy<B2X>(tyy, c2));
      if constexpr (FORM == kSTF2) {
        // kappa grad |grad phi|^2 with |grad phi|^2 = Txx + Tyy at each node
        Fx += P.kappa * (ics_dx<B2X>(txx, c2) + ics_dx<B2X>(tyy, c2));
        Fy += P.kappa * (ics_dy<B2X>(txx, c2) + ics_dy<B2X>(tyy, c2));
      }
    } else if constexpr (FORM == kCPF1) {
      const float* mu = s2 + MU * N2;
      Fx = -phi * ics_dx<B2X>(mu, c2);
      Fy = -phi * ics_dy<B2X>(mu, c2);
    } else if constexpr (FORM == kCPF2) {
      const float mu = s2[MU * N2 + c2];
      Fx = mu * gx;
      Fy = mu * gy;
    } else if constexpr (FORM == kPF1) {
      const float lap = s2[LAP * N2 + c2];
      Fx = -P.kappa * gx * lap;
      Fy = -P.kappa * gy * lap;
    } else if constexpr (FORM == kPF2) {
      const float* lap = s2 + LAP * N2;
      Fx = P.kappa * phi * ics_dx<B2X>(lap, c2);
      Fy = P.kappa * phi * ics_dy<B2X>(lap, c2);
    } else {  // CSF-1, CSF-2
      const float divn = ics_dx<B2X>(s2 + E0 * N2, c2) + ics_dy<B2X>(s2 + (E0 + 1) * N2, c2);
      float coef;
      if constexpr (FORM == kCSF1) coef = -P.kappa * sqrtf(gx * gx + gy * gy) * divn;
      else coef = -P.half_sigma * divn;
      Fx = coef * gx;
      Fy = coef * gy;
    }
    const float rho = P.rho_mid + P.drho_half * phi;
    Fx += (rho - P.rho0) * P.gx;
    Fy += (rho - P.rho0) * P.gy;
    const int gxn = wrap(x0 - 1 + lx, L.nx);
    const int gyn = map_row(y0 - 1 + ly, L.ny, L.wall);
    float f[9];
    pull_f<ST>(a, pull_idx(L, gxn, gyn), f);
    const float jx = (f[1] - f[3]) + ((f[5] - f[6]) + (f[8] - f[7]));
    const float jy = (f[2] - f[4]) + ((f[5] - f[8]) + (f[6] - f[7]));
    // Eq. mac: u = [sum c f + cs^2 F / 2] / (cs^2 rho)
    const float irho = 1.0f / rho;
    const float ux = (3.0f * jx + 0.5f * Fx) * irho;
    const float uy = (3.0f * jy + 0.5f * Fy) * irho;
    s1[FX * N1 + k] = Fx;
    s1[FY * N1 + k] = Fy;
    s1[UX * N1 + k] = ux;
    s1[UY * N1 + k] = uy;
    s1[PUX * N1 + k] = phi * ux;
    s1[PUY * N1 + k] = phi * uy;
  }
  __syncthreads();

  // wall ghosts of phi u: phi (2 u_w - u) of the mirrored node
  if (L.wall) {
    const int lb = -1 - (y0 - 1);      // ring-1 row of y = -1
    const int lt = L.ny - (y0 - 1);    // ring-1 row of y = ny
    const bool bot = lb >= 0 && lb + 1 < B1Y;
    const bool top = lt - 1 >= 0 && lt < B1Y;
    if (bot || top) {
      for (int lx = tid; lx < B1X; lx += kThreads) {
        if (bot) {
          const int g = lb * B1X + lx, m = (lb + 1) * B1X + lx;
          const float pm = sPhi[(lb + 1 + 2) * B3X + lx + 2];
          s1[PUX * N1 + g] = pm * (2.0f * P.uwb - s1[UX * N1 + m]);
          s1[PUY * N1 + g] = -pm * s1[UY * N1 + m];
        }
        if (top) {
          const int g = lt * B1X + lx, m = (lt - 1) * B1X + lx;
          const float pm = sPhi[(lt - 1 + 2) * B3X + lx + 2];
          s1[PUX * N1 + g] = pm * (2.0f * P.uwt - s1[UX * N1 + m]);
          s1[PUY * N1 + g] = -pm * s1[UY * N1 + m];
        }
      }
    }
    __syncthreads();
  }

  // ---- pass 4: collide and store on the tile --------------------------------
  const int nn = L.nx * L.ny;
  for (int k = tid; k < kTX * kTY; k += kThreads) {
    const int ly = k / kTX, lx = k - ly * kTX;
    const int gx = x0 + lx, gy = y0 + ly;
    if (gx >= L.nx || gy >= L.ny) continue;
    const int c1 = (ly + 1) * B1X + lx + 1;
    const int c2 = (ly + 2) * B2X + lx + 2;
    const float phi = sPhi[(ly + 3) * B3X + lx + 3];
    const float Gx = s2[GX * N2 + c2], Gy = s2[GY * N2 + c2];
    const float mu = s2[MU * N2 + c2];
    const float Fx = s1[FX * N1 + c1], Fy = s1[FY * N1 + c1];
    const float ux = s1[UX * N1 + c1], uy = s1[UY * N1 + c1];
    const float rho = P.rho_mid + P.drho_half * phi;
    const float drx = P.drho_half * Gx, dry = P.drho_half * Gy;

    const Pull q = pull_idx(L, gx, gy);
    float f[9];
    pull_f<ST>(a, q, f);
    const float sumf = f[0] + (f[1] + f[2] + f[3] + f[4]) + (f[5] + f[6] + f[7] + f[8]);
    // Eq. mac: P = sum f + cs^2/2 u . grad rho
    const float Pr = sumf + (ux * drx + uy * dry) * (1.0f / 6.0f);
    // div(phi u) by Eq. ICS-1st on the ring-1 values
    const float div = ics_dx<B1X>(s1 + PUX * N1, c1) + ics_dy<B1X>(s1 + PUY * N1, c1);
    const int n_idx = gy * L.nx + gx;
    const float pux = phi * ux, puy = phi * uy;
    float dtx = 0.0f, dty = 0.0f;
    if (!a.first) {
      dtx = pux - a.phiu[n_idx];
      dty = puy - a.phiu[nn + n_idx];
    }

    if (a.macro) {
      const float g2 = Gx * Gx + Gy * Gy;
      const float om = (1.0f - phi) * (1.0f + phi);
      const float f0 = 0.25f * P.beta4 * om * om;
      float ph = Pr;
      if constexpr (FORM == kSTF1) ph = Pr - P.kappa * g2;
      if constexpr (FORM == kCPF1) ph = Pr - f0 + phi * mu + 0.5f * P.kappa * g2;
      if constexpr (FORM == kCPF2) ph = Pr - f0 + 0.5f * P.kappa * g2;
      if constexpr (FORM == kPF1) ph = Pr + 0.5f * P.kappa * g2;
      if constexpr (FORM == kPF2) ph = Pr - P.kappa * phi * s2[LAP * N2 + c2] + 0.5f * P.kappa * g2;
      float* o = a.fields + n_idx;
      o[0 * nn] = phi;
      o[1 * nn] = rho;
      o[2 * nn] = ux;
      o[3 * nn] = uy;
      o[4 * nn] = Pr;
      o[5 * nn] = mu;
      o[6 * nn] = ph;
      o[7 * nn] = Fx;
      o[8 * nn] = Fy;
      continue;
    }
    a.phiu[n_idx] = pux;
    a.phiu[nn + n_idx] = puy;

    float h[9];
    pull_h<ST>(a, q, h);

    // f collision with forcing, Eqs. fh and P_LBM (Gamma_i = w_i (1 + s_i),
    // grad-rho weight w_i s_i)
    const float mv = P.mu_mid + P.mu_dhalf * phi;
    const float tauf = 0.5f + 3.0f * mv * (1.0f / rho);
    const float omf = 1.0f / tauf;
    const float cff = 1.0f - 0.5f * omf;
    const float uu15 = 1.5f * (ux * ux + uy * uy);
    const float uF = ux * Fx + uy * Fy;
    const float rx = drx * (1.0f / 3.0f), ry = dry * (1.0f / 3.0f);
    const float uR = ux * rx + uy * ry;
    const float rho3 = rho * (1.0f / 3.0f);
    // h collision with the CH source, Eqs. fh, heq_CH and CH_LB_force
    const float emu = P.eta * mu;
    const float A = P.acoef * div;
    const float omh = P.inv_tau_h, chh = P.hforce;

    float fo[9], ho[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const float cxi = (float)qcx(i), cyi = (float)qcy(i), wi = qw(i);
      const float cu = cxi * ux + cyi * uy;
      const float s = cu * (3.0f + 4.5f * cu) - uu15;
      const float feq = wi * (Pr + rho3 * s);
      const float Fi = wi * ((1.0f + s) * (cxi * Fx + cyi * Fy - uF) + s * (cxi * rx + cyi * ry - uR));
      fo[i] = f[i] - (f[i] - feq) * omf + cff * Fi;
      float heq, Hi;
      if (i == 0) {
        heq = phi + (wi - 1.0f) * emu;
        Hi = (wi - 1.0f) * A;
      } else {
        heq = wi * (emu + 3.0f * phi * cu);
        Hi = wi * (A + 3.0f * (cxi * dtx + cyi * dty));
      }
      ho[i] = h[i] - (h[i] - heq) * omh + chh * Hi;
    }

    const int o = (gy + 1) * L.nx + gx;
    store_f<ST, 0>(a, o, fo[0]); store_h<ST, 0>(a, o, ho[0]);
    store_f<ST, 1>(a, o, fo[1]); store_h<ST, 1>(a, o, ho[1]);
    store_f<ST, 2>(a, o, fo[2]); store_h<ST, 2>(a, o, ho[2]);
    store_f<ST, 3>(a, o, fo[3]); store_h<ST, 3>(a, o, ho[3]);
    store_f<ST, 4>(a, o, fo[4]); store_h<ST, 4>(a, o, ho[4]);
    store_f<ST, 5>(a, o, fo[5]); store_h<ST, 5>(a, o, ho[5]);
    store_f<ST, 6>(a, o, fo[6]); store_h<ST, 6>(a, o, ho[6]);
    store_f<ST, 7>(a, o, fo[7]); store_h<ST, 7>(a, o, ho[7]);
    store_f<ST, 8>(a, o, fo[8]); store_h<ST, 8>(a, o, ho[8]);

    if (L.wall) {
      // Ladd half-way bounce-back (Sec. 4): a population heading into the
      // wall returns to this node reversed, minus 2 w_i rho c_i.u_w (f) and
      // 2 w_i phi c_i.u_w / cs^2 (h); it is written into the ghost row the
      // next pull reads it from.
      const int xr = gx + 1 < L.nx ? gx + 1 : 0;        // x + 1
      const int xl = gx - 1 >= 0 ? gx - 1 : L.nx - 1;   // x - 1
      if (gy == 0) {
        const float uw = P.uwb;
        // i = 4 (0,-1) -> opp 2 at (x, -1); i = 7 (-1,-1) -> opp 5 at (x-1, -1);
        // i = 8 (1,-1) -> opp 6 at (x+1, -1)
        store_f<ST, 2>(a, gx, fo[4]);
        store_h<ST, 2>(a, gx, ho[4]);
        store_f<ST, 5>(a, xl, fo[7] - 2.0f * qw(7) * rho * (-uw));
        store_h<ST, 5>(a, xl, ho[7] - 2.0f * qw(7) * phi * 3.0f * (-uw));
        store_f<ST, 6>(a, xr, fo[8] - 2.0f * qw(8) * rho * uw);
        store_h<ST, 6>(a, xr, ho[8] - 2.0f * qw(8) * phi * 3.0f * uw);
      }
      if (gy == L.ny - 1) {
        const float uw = P.uwt;
        const int g = (L.ny + 1) * L.nx;
        // i = 2 (0,1) -> opp 4 at (x, ny); i = 5 (1,1) -> opp 7 at (x+1, ny);
        // i = 6 (-1,1) -> opp 8 at (x-1, ny)
        store_f<ST, 4>(a, g + gx, fo[2]);
        store_h<ST, 4>(a, g + gx, ho[2]);
        store_f<ST, 7>(a, g + xr, fo[5] - 2.0f * qw(5) * rho * uw);
        store_h<ST, 7>(a, g + xr, ho[5] - 2.0f * qw(5) * phi * 3.0f * uw);
        store_f<ST, 8>(a, g + xl, fo[6] - 2.0f * qw(6) * rho * (-uw));
        store_h<ST, 8>(a, g + xl, ho[6] - 2.0f * qw(6) * phi * 3.0f * (-uw));
      }
    }
  }
}

template <class ST>
cudaError_t launch_step_impl(int form, const StepArgs& a, cudaStream_t s) {
  dim3 grid((a.L.nx + kTX - 1) / kTX, (a.L.ny + kTY - 1) / kTY);
  switch (form) {
    case kSTF1: k_step<kSTF1, ST><<<grid, kThreads, 0, s>>>(a); break;
    case kSTF2: k_step<kSTF2, ST><<<grid, kThreads, 0, s>>>(a); break;
    case kCPF1: k_step<kCPF1, ST><<<grid, kThreads, 0, s>>>(a); break;
    case kCPF2: k_step<kCPF2, ST><<<grid, kThreads, 0, s>>>(a); break;
    case kPF1: k_step<kPF1, ST><<<grid, kThreads, 0, s>>>(a); break;
    case kPF2: k_step<kPF2, ST><<<grid, kThreads, 0, s>>>(a); break;
    case kCSF1: k_step<kCSF1, ST><<<grid, kThreads, 0, s>>>(a); break;
    case kCSF2: k_step<kCSF2, ST><<<grid, kThreads, 0, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace pflbm

// Fused coupled step of the phase-field lattice Boltzmann method (Sec. 3 of
// Zhang, Liang & Guo, arXiv 2012.14729) for sm_103a.
//
// One CTA owns a kTX x kTY tile of nodes and runs the whole time step for it.
//
// Staging.  The post-collision populations of the previous step are brought
// into shared memory as one 2-D box per population plane: h planes on the
// tile + 3 ring (rows) and f planes on the tile + 1 ring, each box shifted by
// -c_i in y so that its rows hold the pulled values; in x every box spans the
// same 16-byte aligned column range and the -c_ix shift is applied when the
// box is read.  Interior tiles issue the 18 boxes as TMA tensor loads
// (cp.async.bulk.tensor) completing on one mbarrier; tiles whose boxes wrap
// around the periodic seam or reach the wall ghost rows fill the same boxes
// with plain loads.
//
// Passes over shared memory, recomputing the halo a tile's nodes need
// instead of exchanging it through HBM:
//   pass 1  phi = sum_i h_i on the tile + 3 ring (Eq. mac)
//   pass 2  grad phi, lap phi (Eqs. ICS-1st, ICS-sec), mu (Eq.
//           chemical_potential) and the form's level-1 fields on tile + 2
//   pass 3  interfacial + gravity force (Sec. 2.2), rho, u and phi u on
//           tile + 1 (Eq. mac)
//   pass 4  on the tile: P, div(phi u), d_t(phi u), BGK collision of f and h
//           with F_i and H_i (Eqs. fh, P_LBM, CH_LB_force), store of the
//           post-collision populations; streaming is the next step's pull.
// HBM traffic per node and step is the algorithmic state: 18 populations read
// and written plus (phi u) read and written; halo re-reads hit L2.
//
// Walls (Sec. 4, half-way bounce-back): populations are stored with one
// ghost row below and above the domain.  A node next to a wall writes the
// bounced populations (with the moving-wall term) into the ghost row, where
// the next step's pull finds them.  Scalar stencils see mirror ghosts (row
// -k equals row k-1), and the ghost of phi u is phi (2 u_w - u) of the
// mirrored node.
#pragma once

#include "lattice.cuh"

namespace pflbm {

// ---------------------------------------------------------------------------
// TMA and mbarrier (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// 2-D tensor tile load global -> shared, completion counted on `bar`.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

// ---------------------------------------------------------------------------
// shared-memory geometry of one CTA
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int pad128(int b) { return (b + 127) / 128 * 128; }

template <class ST, int FORM>
struct Smem {
  using T = typename ST::T;
  static constexpr int EB = sizeof(T);
  static constexpr int XPAD = box_xpad(EB);
  static constexpr int PW = box_w(EB);
  static constexpr int RH = kBoxRowsH, RF = kBoxRowsF;
  // boxes: h planes (h_0 in float32 when the storage is split), f planes
  static constexpr int HB0 = pad128(RH * PW * (ST::kSplitH0 ? 4 : EB));
  static constexpr int HB = pad128(RH * PW * EB);
  static constexpr int FB = pad128(RF * PW * EB);
  static constexpr int B3X = kTX + 6, B3Y = kTY + 6;
  static constexpr int B2X = kTX + 4, B2Y = kTY + 4;
  static constexpr int B1X = kTX + 2, B1Y = kTY + 2;
  static constexpr int N3 = B3X * B3Y, N2 = B2X * B2Y, N1 = B1X * B1Y;
  static constexpr int NE = extra_fields<FORM>();
  static constexpr int OFF_BAR = 0;
  static constexpr int OFF_H = 128;
  static constexpr int OFF_F = OFF_H + HB0 + 8 * HB;
  static constexpr int OFF_PHI = OFF_F + 9 * FB;
  static constexpr int OFF_S2 = OFF_PHI + pad128(N3 * 4);
  static constexpr int OFF_S1 = OFF_S2 + pad128((4 + NE) * N2 * 4);
  static constexpr int BYTES = OFF_S1 + pad128(6 * N1 * 4);
  static constexpr int TMA_BYTES = HB0 + 8 * HB + 9 * FB;  // counted per box, padded
  static constexpr int TMA_TX = RH * PW * (ST::kSplitH0 ? 4 : EB) + 8 * RH * PW * EB +
                                9 * RF * PW * EB;  // bytes the 18 loads deliver

  __device__ static int h_off(int i) { return OFF_H + (i == 0 ? 0 : HB0 + (i - 1) * HB); }
  __device__ static int f_off(int i) { return OFF_F + i * FB; }
};

// population i of a box at (row, col), decoded to float
template <class ST, int I, class G>
__device__ __forceinline__ float box_h(const unsigned char* sm, int r, int c, const Phys& P) {
  if constexpr (ST::kSplitH0 && I == 0) {
    return reinterpret_cast<const float*>(sm + G::h_off(0))[r * G::PW + c];
  } else {
    const typename ST::T v = reinterpret_cast<const typename ST::T*>(sm + G::h_off(I))[r * G::PW + c];
    return ST::dec(v, qw(I) * P.inv_sh);
  }
}
template <class ST, int I, class G>
__device__ __forceinline__ float box_f(const unsigned char* sm, int r, int c, const Phys& P) {
  const typename ST::T v = reinterpret_cast<const typename ST::T*>(sm + G::f_off(I))[r * G::PW + c];
  return ST::dec(v, qw(I) * P.inv_sf);
}

// Fill the boxes with plain loads (tiles at the periodic seam or the walls).
// Box row r of plane i holds storage row (node row - c_iy) + 1 of the rows
// the tile needs; rows the tile never pulls (beyond a wall) are zero.
template <class ST, class G>
__device__ void fill_boxes_plain(const StepArgs& a, unsigned char* sm, int x0, int y0) {
  using T = typename ST::T;
  const Lattice& L = a.L;
  auto srow = [&](int yy) -> int {  // storage row of source domain row yy, or -1
    if (L.wall) return (yy >= -1 && yy <= L.ny) ? yy + 1 : -1;
    return wrap(yy, L.ny) + 1;
  };
  for (int e = threadIdx.x; e < G::RH * G::PW; e += kThreads) {
    const int r = e / G::PW, c = e - r * G::PW;
    const int gx = wrap(x0 - G::XPAD + c, L.nx);
    const int yn = y0 - 3 + r;  // node row
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int sr = srow(yn - qcy(i));
      if (ST::kSplitH0 && i == 0) {
        reinterpret_cast<float*>(sm + G::h_off(0))[e] = sr >= 0 ? a.h0_in[sr * L.nx + gx] : 0.0f;
      } else {
        const int pl = ST::kSplitH0 ? i - 1 : i;
        const T* src = reinterpret_cast<const T*>(a.h_in) + (size_t)pl * L.plane;
        reinterpret_cast<T*>(sm + G::h_off(i))[e] = sr >= 0 ? src[sr * L.nx + gx] : T(0.0f);
      }
    }
  }
  for (int e = threadIdx.x; e < G::RF * G::PW; e += kThreads) {
    const int r = e / G::PW, c = e - r * G::PW;
    const int gx = wrap(x0 - G::XPAD + c, L.nx);
    const int yn = y0 - 1 + r;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int sr = srow(yn - qcy(i));
      const T* src = reinterpret_cast<const T*>(a.f_in) + (size_t)i * L.plane;
      reinterpret_cast<T*>(sm + G::f_off(i))[e] = sr >= 0 ? src[sr * L.nx + gx] : T(0.0f);
    }
  }
}

// ---------------------------------------------------------------------------
// the fused step kernel
// ---------------------------------------------------------------------------
template <int FORM, class ST>
__global__ void __launch_bounds__(kThreads, 2) k_step(const __grid_constant__ StepArgs a) {
  using G = Smem<ST, FORM>;
  constexpr int B3X = G::B3X, B2X = G::B2X, B1X = G::B1X, B1Y = G::B1Y;
  constexpr int N2 = G::N2, N1 = G::N1;
  constexpr int PW = G::PW, XP = G::XPAD;
  // level-1 field slots in s2, ring-1 slots in s1
  constexpr int GX = 0, GY = 1, LAP = 2, MU = 3, E0 = 4;
  constexpr int FX = 0, FY = 1, UX = 2, UY = 3, PUX = 4, PUY = 5;

  extern __shared__ __align__(128) unsigned char sm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + G::OFF_BAR);
  float* sPhi = reinterpret_cast<float*>(sm + G::OFF_PHI);
  float* s2 = reinterpret_cast<float*>(sm + G::OFF_S2);
  float* s1 = reinterpret_cast<float*>(sm + G::OFF_S1);

  const Lattice L = a.L;
  const Phys& P = a.p;
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
  const int tid = threadIdx.x;

  // ---- staging ---------------------------------------------------------------
  const bool tma = a.use_tma && x0 - XP >= 0 && x0 + kTX + XP <= L.nx && y0 >= 4 &&
                   y0 + kTY + 4 <= L.ny;
  if (tma) {
    if (tid == 0) {
      mbar_init(bar, 1);
      fence_mbar_init();
      mbar_arrive_expect_tx(bar, G::TMA_TX);
      const int xs = x0 - XP;
      const int rows = L.ny + 2;
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        // h box of plane i: storage rows from (y0 - 3 - c_iy) + 1
        const int yh = y0 - 2 - qcy(i);
        if (ST::kSplitH0 && i == 0) tma_load_2d(sm + G::h_off(0), &a.tm_h0, xs, yh, bar);
        else tma_load_2d(sm + G::h_off(i), &a.tm_h, xs, (ST::kSplitH0 ? i - 1 : i) * rows + yh, bar);
        // f box of plane i: storage rows from (y0 - 1 - c_iy) + 1
        tma_load_2d(sm + G::f_off(i), &a.tm_f, xs, i * rows + y0 - qcy(i), bar);
      }
    }
    __syncthreads();  // barrier initialised before anyone waits on it
    int timed_out = 0;
    for (long long n = 0; !mbar_try_wait(bar, 0);) {
      if (++n > kWaitLimit) {
        timed_out = 1;
        break;
      }
    }
    if (__syncthreads_or(timed_out)) {
      // the loads did not complete: flag it, wait (bounded) for the copies
      // still in flight so none lands after the CTA exits, and give up
      if (tid == 0) atomicOr(a.err, 1);
      for (long long m = 0; m < kWaitLimit && !mbar_try_wait(bar, 0); ++m) {
      }
      return;
    }
  } else {
    fill_boxes_plain<ST, G>(a, sm, x0, y0);
    __syncthreads();
  }

  // ---- pass 1: phi on tile + 3 ------------------------------------------------
  for (int k = tid; k < G::N3; k += kThreads) {
    const int r = k / B3X, cc = k - r * B3X;
    const int yn = y0 - 3 + r;
    if (L.wall && (yn < 0 || yn >= L.ny)) continue;  // mirrored below
    const int c = cc + XP - 3;
    float s = box_h<ST, 0, G>(sm, r, c, P);
    s += box_h<ST, 1, G>(sm, r, c - 1, P);
    s += box_h<ST, 2, G>(sm, r, c, P);
    s += box_h<ST, 3, G>(sm, r, c + 1, P);
    s += box_h<ST, 4, G>(sm, r, c, P);
    s += box_h<ST, 5, G>(sm, r, c - 1, P);
    s += box_h<ST, 6, G>(sm, r, c + 1, P);
    s += box_h<ST, 7, G>(sm, r, c + 1, P);
    s += box_h<ST, 8, G>(sm, r, c - 1, P);
    sPhi[k] = s;
  }
  __syncthreads();
  if (L.wall && (y0 - 3 < 0 || y0 + kTY + 3 > L.ny)) {
    // mirror ghosts of phi about the wall planes
    for (int k = tid; k < G::N3; k += kThreads) {
      const int r = k / B3X, cc = k - r * B3X;
      const int yn = y0 - 3 + r;
      if (yn >= 0 && yn < L.ny) continue;
      const int rm = map_row(yn, L.ny, 1) - (y0 - 3);
      sPhi[k] = (rm >= 0 && rm < G::B3Y) ? sPhi[rm * B3X + cc] : 0.0f;
    }
    __syncthreads();
  }

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
    // pulled f from the boxes: row ly, column (lx - 1) + XP - c_ix
    const int c = lx + XP - 1;
    const float f1 = box_f<ST, 1, G>(sm, ly, c - 1, P), f2 = box_f<ST, 2, G>(sm, ly, c, P);
    const float f3 = box_f<ST, 3, G>(sm, ly, c + 1, P), f4 = box_f<ST, 4, G>(sm, ly, c, P);
    const float f5 = box_f<ST, 5, G>(sm, ly, c - 1, P), f6 = box_f<ST, 6, G>(sm, ly, c + 1, P);
    const float f7 = box_f<ST, 7, G>(sm, ly, c + 1, P), f8 = box_f<ST, 8, G>(sm, ly, c - 1, P);
    const float jx = (f1 - f3) + ((f5 - f6) + (f8 - f7));
    const float jy = (f2 - f4) + ((f5 - f8) + (f6 - f7));
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

    // pulled populations: f box row ly + 1, h box row ly + 3, column lx + XP - c_ix
    const int c = lx + XP;
    float f[9];
    f[0] = box_f<ST, 0, G>(sm, ly + 1, c, P);
    f[1] = box_f<ST, 1, G>(sm, ly + 1, c - 1, P);
    f[2] = box_f<ST, 2, G>(sm, ly + 1, c, P);
    f[3] = box_f<ST, 3, G>(sm, ly + 1, c + 1, P);
    f[4] = box_f<ST, 4, G>(sm, ly + 1, c, P);
    f[5] = box_f<ST, 5, G>(sm, ly + 1, c - 1, P);
    f[6] = box_f<ST, 6, G>(sm, ly + 1, c + 1, P);
    f[7] = box_f<ST, 7, G>(sm, ly + 1, c + 1, P);
    f[8] = box_f<ST, 8, G>(sm, ly + 1, c - 1, P);
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
    h[0] = box_h<ST, 0, G>(sm, ly + 3, c, P);
    h[1] = box_h<ST, 1, G>(sm, ly + 3, c - 1, P);
    h[2] = box_h<ST, 2, G>(sm, ly + 3, c, P);
    h[3] = box_h<ST, 3, G>(sm, ly + 3, c + 1, P);
    h[4] = box_h<ST, 4, G>(sm, ly + 3, c, P);
    h[5] = box_h<ST, 5, G>(sm, ly + 3, c - 1, P);
    h[6] = box_h<ST, 6, G>(sm, ly + 3, c + 1, P);
    h[7] = box_h<ST, 7, G>(sm, ly + 3, c + 1, P);
    h[8] = box_h<ST, 8, G>(sm, ly + 3, c - 1, P);

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

template <int FORM, class ST>
cudaError_t launch_form(const StepArgs& a, cudaStream_t s) {
  using G = Smem<ST, FORM>;
  static bool configured = false;  // per instantiation; attribute is per device function
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_step<FORM, ST>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, G::BYTES);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  dim3 grid((a.L.nx + kTX - 1) / kTX, (a.L.ny + kTY - 1) / kTY);
  k_step<FORM, ST><<<grid, kThreads, G::BYTES, s>>>(a);
  return cudaGetLastError();
}

template <class ST>
cudaError_t launch_step_impl(int form, const StepArgs& a, cudaStream_t s) {
  switch (form) {
    case kSTF1: return launch_form<kSTF1, ST>(a, s);
    case kSTF2: return launch_form<kSTF2, ST>(a, s);
    case kCPF1: return launch_form<kCPF1, ST>(a, s);
    case kCPF2: return launch_form<kCPF2, ST>(a, s);
    case kPF1: return launch_form<kPF1, ST>(a, s);
    case kPF2: return launch_form<kPF2, ST>(a, s);
    case kCSF1: return launch_form<kCSF1, ST>(a, s);
    case kCSF2: return launch_form<kCSF2, ST>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pflbm

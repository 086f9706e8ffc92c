// Fused coupled step of the phase-field lattice Boltzmann method (Sec. 3 of
// Zhang, Liang & Guo, arXiv 2012.14729) for sm_103a.
//
// A persistent kernel: one 512-thread CTA per SM walks a list of kTX x kTY
// tiles and runs the whole time step for each.
//
// Staging.  The post-collision populations of the previous step are brought
// into shared memory as one 2-D box per population plane: h planes on the
// tile + 3 ring (rows) and f planes on the tile + 1 ring, each box shifted by
// -c_i in y so that its rows hold the pulled values; in x every box spans the
// same 16-byte aligned column range and the -c_ix shift is applied when the
// box is read.  Interior tiles issue their 18 boxes as TMA tensor loads
// (cp.async.bulk.tensor) completing on an mbarrier.  Two box buffers
// alternate: while a CTA computes one tile, the TMA loads of its next tile
// are in flight.  Tiles whose boxes wrap around the periodic seam or reach
// the wall ghost rows fill the same boxes with plain loads.
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
// order this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy (TMA) writes to it
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
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
  static constexpr int BUF = HB0 + 8 * HB + 9 * FB;  // one set of 18 boxes
  static constexpr int B3X = kTX + 6, B3Y = kTY + 6;
  static constexpr int B2X = kTX + 4, B2Y = kTY + 4;
  static constexpr int B1X = kTX + 2, B1Y = kTY + 2;
  static constexpr int N3 = B3X * B3Y, N2 = B2X * B2Y, N1 = B1X * B1Y;
  static constexpr int NE = extra_fields<FORM>();
  static constexpr int OFF_BAR = 0;        // two mbarriers
  static constexpr int OFF_BUF = 128;      // two box buffers
  static constexpr int OFF_PHI = OFF_BUF + kBoxBuffers * BUF;
  static constexpr int OFF_S2 = OFF_PHI + pad128(N3 * 4);
  static constexpr int OFF_S1 = OFF_S2 + pad128((4 + NE) * N2 * 4);
  static constexpr int BYTES = OFF_S1 + pad128(6 * N1 * 4);
  static constexpr int TMA_TX = RH * PW * (ST::kSplitH0 ? 4 : EB) + 8 * RH * PW * EB +
                                9 * RF * PW * EB;  // bytes the 18 loads deliver

  __device__ static int h_off(int i) { return i == 0 ? 0 : HB0 + (i - 1) * HB; }
  __device__ static int f_off(int i) { return HB0 + 8 * HB + i * FB; }
};

// population i of a box set at (row, col), decoded to float
template <class ST, int I, class G>
__device__ __forceinline__ float box_h(const unsigned char* bx, int r, int c, const Phys& P) {
  if constexpr (ST::kSplitH0 && I == 0) {
    return reinterpret_cast<const float*>(bx + G::h_off(0))[r * G::PW + c];
  } else {
    const typename ST::T v =
        reinterpret_cast<const typename ST::T*>(bx + G::h_off(I))[r * G::PW + c];
    return ST::dec(v, qw(I) * P.inv_sh);
  }
}
template <class ST, int I, class G>
__device__ __forceinline__ float box_f(const unsigned char* bx, int r, int c, const Phys& P) {
  const typename ST::T v = reinterpret_cast<const typename ST::T*>(bx + G::f_off(I))[r * G::PW + c];
  return ST::dec(v, qw(I) * P.inv_sf);
}

// Tiles whose 18 boxes lie inside the stored planes without wrapping.
template <class G>
__device__ __forceinline__ bool tma_tile(const StepArgs& a, int x0, int y0) {
  return a.use_tma && x0 - G::XPAD >= 0 && x0 + kTX + G::XPAD <= a.L.nx && y0 >= 4 &&
         y0 + kTY + 4 <= a.L.ny;
}

// Issue the 18 box loads of the tile at (x0, y0) into box set bx (one thread).
template <class ST, class G>
__device__ __forceinline__ void issue_tma(const StepArgs& a, unsigned char* bx, uint64_t* bar,
                                          int x0, int y0) {
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(bar, G::TMA_TX);
  const int xs = x0 - G::XPAD;
  const int rows = a.L.ny + 2;
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    // h box of plane i: storage rows from (y0 - 3 - c_iy) + 1
    const int yh = y0 - 2 - qcy(i);
    if (ST::kSplitH0 && i == 0) tma_load_2d(bx + G::h_off(0), &a.tm_h0, xs, yh, bar);
    else tma_load_2d(bx + G::h_off(i), &a.tm_h, xs, (ST::kSplitH0 ? i - 1 : i) * rows + yh, bar);
    // f box of plane i: storage rows from (y0 - 1 - c_iy) + 1
    tma_load_2d(bx + G::f_off(i), &a.tm_f, xs, i * rows + y0 - qcy(i), bar);
  }
}

// Fill the boxes with plain loads (tiles at the periodic seam or the walls).
// Box row r of plane i holds storage row (node row - c_iy) + 1 of the rows
// the tile needs; rows the tile never pulls (beyond a wall) are zero.
template <class ST, class G>
__device__ void fill_boxes_plain(const StepArgs& a, unsigned char* bx, int x0, int y0) {
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
        reinterpret_cast<float*>(bx + G::h_off(0))[e] = sr >= 0 ? a.h0_in[sr * L.nx + gx] : 0.0f;
      } else {
        const int pl = ST::kSplitH0 ? i - 1 : i;
        const T* src = reinterpret_cast<const T*>(a.h_in) + (size_t)pl * L.plane;
        reinterpret_cast<T*>(bx + G::h_off(i))[e] = sr >= 0 ? src[sr * L.nx + gx] : T(0.0f);
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
      reinterpret_cast<T*>(bx + G::f_off(i))[e] = sr >= 0 ? src[sr * L.nx + gx] : T(0.0f);
    }
  }
}

// Asynchronous version of fill_boxes_plain for 4-byte storage: each element
// is one cp.async (zero-filled when the source row is beyond a wall), so
// seam and wall tiles are prefetched like TMA tiles.  Completion: each
// thread's cp.async.wait_all, then a CTA barrier.
__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_addr(dst)), "l"(src),
               "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}
template <class ST, class G>
__device__ void fill_boxes_async(const StepArgs& a, unsigned char* bx, int x0, int y0) {
  static_assert(sizeof(typename ST::T) == 4, "cp.async path is for 4-byte storage");
  const Lattice& L = a.L;
  auto srow = [&](int yy) -> int {
    if (L.wall) return (yy >= -1 && yy <= L.ny) ? yy + 1 : -1;
    return wrap(yy, L.ny) + 1;
  };
  const float* hin = reinterpret_cast<const float*>(a.h_in);
  const float* fin = reinterpret_cast<const float*>(a.f_in);
  for (int e = threadIdx.x; e < G::RH * G::PW; e += kThreads) {
    const int r = e / G::PW, c = e - r * G::PW;
    const int gx = wrap(x0 - G::XPAD + c, L.nx);
    const int yn = y0 - 3 + r;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int sr = srow(yn - qcy(i));
      const float* src = hin + (size_t)i * L.plane + (sr >= 0 ? sr * L.nx + gx : 0);
      cp_async4(reinterpret_cast<float*>(bx + G::h_off(i)) + e, src, sr >= 0);
    }
  }
  for (int e = threadIdx.x; e < G::RF * G::PW; e += kThreads) {
    const int r = e / G::PW, c = e - r * G::PW;
    const int gx = wrap(x0 - G::XPAD + c, L.nx);
    const int yn = y0 - 1 + r;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int sr = srow(yn - qcy(i));
      const float* src = fin + (size_t)i * L.plane + (sr >= 0 ? sr * L.nx + gx : 0);
      cp_async4(reinterpret_cast<float*>(bx + G::f_off(i)) + e, src, sr >= 0);
    }
  }
}

// Bounded wait for a box set; returns false (after flagging a.err and a
// second bounded wait for copies still in flight) if it did not complete.
__device__ __forceinline__ bool wait_boxes(const StepArgs& a, uint64_t* bar, uint32_t parity) {
  int timed_out = 0;
  for (long long n = 0; !mbar_try_wait(bar, parity);) {
    if (++n > kWaitLimit) {
      timed_out = 1;
      break;
    }
  }
  if (__syncthreads_or(timed_out)) {
    if (threadIdx.x == 0) atomicOr(a.err, 1);
    for (long long m = 0; m < kWaitLimit && !mbar_try_wait(bar, parity); ++m) {
    }
    return false;
  }
  return true;
}

// One collision of an opposite pair (i, j) with c_j = -c_i, w_j = w_i:
// f_i^+ = f_i (1 - 1/tau_f) + f_i^eq / tau_f + (1 - 1/(2 tau_f)) F_i and the
// same for h with tau_h and H_i (Eqs. fh, P_LBM, CH_LB_force, heq_CH).
struct CollideConsts {
  float ux, uy, Pr, rho3, uu15, Fx, Fy, uF, rx, ry, uR, omf, omf1, cff;
  float phi3, emu, A, dtx, dty, omh, omh1, chh;
};
template <int I>
__device__ __forceinline__ void collide_pair(const CollideConsts& k, float fi, float fj, float hi,
                                             float hj, float& foi, float& foj, float& hoi,
                                             float& hoj) {
  constexpr float w = qw(I);
  constexpr float cx = (float)qcx(I), cy = (float)qcy(I);
  const float cu = cx * k.ux + cy * k.uy;
  const float l = 3.0f * cu;
  const float q = 4.5f * cu * cu - k.uu15;
  const float si = q + l, sj = q - l;
  const float cF = cx * k.Fx + cy * k.Fy;
  const float cR = cx * k.rx + cy * k.ry;
  const float feqi = w * (k.Pr + k.rho3 * si);
  const float feqj = w * (k.Pr + k.rho3 * sj);
  const float Fi = w * ((1.0f + si) * (cF - k.uF) + si * (cR - k.uR));
  const float Fj = w * ((1.0f + sj) * (-cF - k.uF) + sj * (-cR - k.uR));
  foi = fi * k.omf1 + feqi * k.omf + k.cff * Fi;
  foj = fj * k.omf1 + feqj * k.omf + k.cff * Fj;
  const float hc = k.phi3 * cu;
  const float cdt = 3.0f * (cx * k.dtx + cy * k.dty);
  const float heqi = w * (k.emu + hc), heqj = w * (k.emu - hc);
  const float Hi = w * (k.A + cdt), Hj = w * (k.A - cdt);
  hoi = hi * k.omh1 + heqi * k.omh + k.chh * Hi;
  hoj = hj * k.omh1 + heqj * k.omh + k.chh * Hj;
}

// ---------------------------------------------------------------------------
// one tile: passes 1-4 from the box set bx
// ---------------------------------------------------------------------------
template <int FORM, class ST>
__device__ __forceinline__ void step_tile(const StepArgs& a, const unsigned char* bx,
                                          unsigned char* sm, int x0, int y0) {
  using G = Smem<ST, FORM>;
  constexpr int B3X = G::B3X, B2X = G::B2X, B1X = G::B1X, B1Y = G::B1Y;
  constexpr int N2 = G::N2, N1 = G::N1;
  constexpr int XP = G::XPAD;
  // level-1 field slots in s2, ring-1 slots in s1
  constexpr int GX = 0, GY = 1, LAP = 2, MU = 3, E0 = 4;
  constexpr int FX = 0, FY = 1, UX = 2, UY = 3, PUX = 4, PUY = 5;
  float* sPhi = reinterpret_cast<float*>(sm + G::OFF_PHI);
  float* s2 = reinterpret_cast<float*>(sm + G::OFF_S2);
  float* s1 = reinterpret_cast<float*>(sm + G::OFF_S1);
  const Lattice& L = a.L;
  const Phys& P = a.p;
  const int tid = threadIdx.x;
  static_assert(kTX * kTY == kThreads, "one collision node per thread");

  // (phi u)^{t-1} of this thread's collision node, loaded first so that the
  // load latency overlaps passes 1-3
  const int nn = L.nx * L.ny;
  float pu_prev_x = 0.0f, pu_prev_y = 0.0f;
  {
    const int gx = x0 + tid % kTX, gy = y0 + tid / kTX;
    if (!a.first && !a.macro && gx < L.nx && gy < L.ny) {
      pu_prev_x = a.phiu[gy * L.nx + gx];
      pu_prev_y = a.phiu[nn + gy * L.nx + gx];
    }
  }

  // ---- pass 1: phi on tile + 3 ------------------------------------------------
  for (int k = tid; k < G::N3; k += kThreads) {
    const int r = k / B3X, cc = k - r * B3X;
    const int yn = y0 - 3 + r;
    if (L.wall && (yn < 0 || yn >= L.ny)) continue;  // mirrored below
    const int c = cc + XP - 3;
    float s = box_h<ST, 0, G>(bx, r, c, P);
    s += box_h<ST, 1, G>(bx, r, c - 1, P);
    s += box_h<ST, 2, G>(bx, r, c, P);
    s += box_h<ST, 3, G>(bx, r, c + 1, P);
    s += box_h<ST, 4, G>(bx, r, c, P);
    s += box_h<ST, 5, G>(bx, r, c - 1, P);
    s += box_h<ST, 6, G>(bx, r, c + 1, P);
    s += box_h<ST, 7, G>(bx, r, c + 1, P);
    s += box_h<ST, 8, G>(bx, r, c - 1, P);
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
    const float f1 = box_f<ST, 1, G>(bx, ly, c - 1, P), f2 = box_f<ST, 2, G>(bx, ly, c, P);
    const float f3 = box_f<ST, 3, G>(bx, ly, c + 1, P), f4 = box_f<ST, 4, G>(bx, ly, c, P);
    const float f5 = box_f<ST, 5, G>(bx, ly, c - 1, P), f6 = box_f<ST, 6, G>(bx, ly, c + 1, P);
    const float f7 = box_f<ST, 7, G>(bx, ly, c + 1, P), f8 = box_f<ST, 8, G>(bx, ly, c - 1, P);
    const float jx = (f1 - f3) + ((f5 - f6) + (f8 - f7));
    const float jy = (f2 - f4) + ((f5 - f8) + (f6 - f7));
    // Eq. mac: u = [sum c f + cs^2 F / 2] / (cs^2 rho)
    const float irho = __fdividef(1.0f, rho);
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
    const float f0 = box_f<ST, 0, G>(bx, ly + 1, c, P);
    const float f1 = box_f<ST, 1, G>(bx, ly + 1, c - 1, P);
    const float f2 = box_f<ST, 2, G>(bx, ly + 1, c, P);
    const float f3 = box_f<ST, 3, G>(bx, ly + 1, c + 1, P);
    const float f4 = box_f<ST, 4, G>(bx, ly + 1, c, P);
    const float f5 = box_f<ST, 5, G>(bx, ly + 1, c - 1, P);
    const float f6 = box_f<ST, 6, G>(bx, ly + 1, c + 1, P);
    const float f7 = box_f<ST, 7, G>(bx, ly + 1, c + 1, P);
    const float f8 = box_f<ST, 8, G>(bx, ly + 1, c - 1, P);
    const float sumf = f0 + (f1 + f2 + f3 + f4) + (f5 + f6 + f7 + f8);
    // Eq. mac: P = sum f + cs^2/2 u . grad rho
    const float Pr = sumf + (ux * drx + uy * dry) * (1.0f / 6.0f);
    // div(phi u) by Eq. ICS-1st on the ring-1 values
    const float div = ics_dx<B1X>(s1 + PUX * N1, c1) + ics_dy<B1X>(s1 + PUY * N1, c1);
    const int n_idx = gy * L.nx + gx;
    const float pux = phi * ux, puy = phi * uy;
    float dtx = 0.0f, dty = 0.0f;
    if (!a.first) {
      dtx = pux - pu_prev_x;
      dty = puy - pu_prev_y;
    }

    if (a.macro) {
      const float g2 = Gx * Gx + Gy * Gy;
      const float om = (1.0f - phi) * (1.0f + phi);
      const float f0e = 0.25f * P.beta4 * om * om;
      float ph = Pr;
      if constexpr (FORM == kSTF1) ph = Pr - P.kappa * g2;
      if constexpr (FORM == kCPF1) ph = Pr - f0e + phi * mu + 0.5f * P.kappa * g2;
      if constexpr (FORM == kCPF2) ph = Pr - f0e + 0.5f * P.kappa * g2;
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

    const float h0 = box_h<ST, 0, G>(bx, ly + 3, c, P);
    const float h1 = box_h<ST, 1, G>(bx, ly + 3, c - 1, P);
    const float h2 = box_h<ST, 2, G>(bx, ly + 3, c, P);
    const float h3 = box_h<ST, 3, G>(bx, ly + 3, c + 1, P);
    const float h4 = box_h<ST, 4, G>(bx, ly + 3, c, P);
    const float h5 = box_h<ST, 5, G>(bx, ly + 3, c - 1, P);
    const float h6 = box_h<ST, 6, G>(bx, ly + 3, c + 1, P);
    const float h7 = box_h<ST, 7, G>(bx, ly + 3, c + 1, P);
    const float h8 = box_h<ST, 8, G>(bx, ly + 3, c - 1, P);

    // relaxation constants: tau_f = 1/2 + mu(phi) / (cs^2 rho) (Sec. 3)
    const float mv = P.mu_mid + P.mu_dhalf * phi;
    const float omf = __fdividef(1.0f, 0.5f + 3.0f * mv * __fdividef(1.0f, rho));
    CollideConsts K;
    K.ux = ux;
    K.uy = uy;
    K.Pr = Pr;
    K.rho3 = rho * (1.0f / 3.0f);
    K.uu15 = 1.5f * (ux * ux + uy * uy);
    K.Fx = Fx;
    K.Fy = Fy;
    K.uF = ux * Fx + uy * Fy;
    K.rx = drx * (1.0f / 3.0f);
    K.ry = dry * (1.0f / 3.0f);
    K.uR = ux * K.rx + uy * K.ry;
    K.omf = omf;
    K.omf1 = 1.0f - omf;
    K.cff = 1.0f - 0.5f * omf;
    K.phi3 = 3.0f * phi;
    K.emu = P.eta * mu;
    K.A = P.acoef * div;
    K.dtx = dtx;
    K.dty = dty;
    K.omh = P.inv_tau_h;
    K.omh1 = 1.0f - P.inv_tau_h;
    K.chh = P.hforce;

    float fo[9], ho[9];
    {
      // rest population: s_0 = -1.5 |u|^2, c_0 = 0, wbar_0 = w_0 - 1
      constexpr float w0 = qw(0);
      const float s0 = -K.uu15;
      const float feq0 = w0 * (Pr + K.rho3 * s0);
      const float F0 = w0 * ((1.0f + s0) * (-K.uF) + s0 * (-K.uR));
      fo[0] = f0 * K.omf1 + feq0 * omf + K.cff * F0;
      const float heq0 = phi + (w0 - 1.0f) * K.emu;
      ho[0] = h0 * K.omh1 + heq0 * K.omh + K.chh * ((w0 - 1.0f) * K.A);
    }
    collide_pair<1>(K, f1, f3, h1, h3, fo[1], fo[3], ho[1], ho[3]);
    collide_pair<2>(K, f2, f4, h2, h4, fo[2], fo[4], ho[2], ho[4]);
    collide_pair<5>(K, f5, f7, h5, h7, fo[5], fo[7], ho[5], ho[7]);
    collide_pair<6>(K, f6, f8, h6, h8, fo[6], fo[8], ho[6], ho[8]);

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

// ---------------------------------------------------------------------------
// the persistent step kernel
// ---------------------------------------------------------------------------
template <int FORM, class ST>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_step(const __grid_constant__ StepArgs a) {
  using G = Smem<ST, FORM>;
  extern __shared__ __align__(128) unsigned char sm[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + G::OFF_BAR);
  unsigned char* bufs = sm + G::OFF_BUF;

  const int ntx = (a.L.nx + kTX - 1) / kTX;
  const int ntiles = ntx * ((a.L.ny + kTY - 1) / kTY);
  int t = blockIdx.x;
  if (t >= ntiles) return;
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  __syncthreads();

  // seam and wall tiles of 4-byte storage are prefetched with cp.async;
  // for 16-bit storage they are filled synchronously before use
  constexpr bool kAsyncFill = sizeof(typename ST::T) == 4;
  uint32_t parity = 0u;
  int buf = 0;
  int x0 = (t % ntx) * kTX, y0 = (t / ntx) * kTY;
  bool tma_cur = tma_tile<G>(a, x0, y0);
  if (tma_cur) {
    if (threadIdx.x == 0) issue_tma<ST, G>(a, bufs, &bars[0], x0, y0);
  } else if constexpr (kAsyncFill) {
    fill_boxes_async<ST, G>(a, bufs, x0, y0);
  } else {
    fill_boxes_plain<ST, G>(a, bufs, x0, y0);
    __syncthreads();
  }

  for (;;) {
    unsigned char* bx = bufs + buf * G::BUF;
    if (tma_cur) {
      // phase parity of each buffer's barrier, kept in two bits of `parity`
      if (!wait_boxes(a, &bars[buf], (parity >> buf) & 1u)) return;
      parity ^= 1u << buf;
    } else if constexpr (kAsyncFill) {
      cp_async_wait_all();
      __syncthreads();
    }
    const int tn = t + gridDim.x;
    const int xn = (tn % ntx) * kTX, yn = (tn / ntx) * kTY;
    const bool tma_next = tn < ntiles && tma_tile<G>(a, xn, yn);
    const int nb = kBoxBuffers == 2 ? buf ^ 1 : 0;  // buffer of the next tile
    if constexpr (kBoxBuffers == 2) {
      // prefetch the next tile into the other buffer (its last reader, the
      // tile before this one, finished at the barrier closing that tile)
      if (tma_next) {
        if (threadIdx.x == 0) issue_tma<ST, G>(a, bufs + nb * G::BUF, &bars[nb], xn, yn);
      } else if constexpr (kAsyncFill) {
        if (tn < ntiles) fill_boxes_async<ST, G>(a, bufs + nb * G::BUF, xn, yn);
      }
    }

    step_tile<FORM, ST>(a, bx, sm, x0, y0);
    __syncthreads();

    if (tn >= ntiles) break;
    if constexpr (kBoxBuffers == 1) {
      // single buffer: stage the next tile now that this one is done
      if (tma_next) {
        if (threadIdx.x == 0) issue_tma<ST, G>(a, bufs, &bars[0], xn, yn);
      } else if constexpr (kAsyncFill) {
        fill_boxes_async<ST, G>(a, bufs, xn, yn);
      } else {
        fill_boxes_plain<ST, G>(a, bufs, xn, yn);
        __syncthreads();
      }
    } else if constexpr (!kAsyncFill) {
      if (!tma_next) {
        fill_boxes_plain<ST, G>(a, bufs + nb * G::BUF, xn, yn);
        __syncthreads();
      }
    }
    t = tn;
    x0 = xn;
    y0 = yn;
    tma_cur = tma_next;
    buf = nb;
  }
}

int num_sms();

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
  const int ntiles = ((a.L.nx + kTX - 1) / kTX) * ((a.L.ny + kTY - 1) / kTY);
  const int slots = num_sms() * kMinBlocks;
  const int grid = ntiles < slots ? ntiles : slots;
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

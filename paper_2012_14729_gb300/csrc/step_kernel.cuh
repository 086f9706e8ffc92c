// Fused coupled step of the phase-field lattice Boltzmann method (Sec. 3 of
// Zhang, Liang & Guo, arXiv 2012.14729) for sm_103a.
//
// A CTA runs the whole time step for kTX x kTY tiles of nodes, in passes over
// shared memory that recompute the halo a tile's nodes need instead of
// exchanging it through HBM:
//   pass 1  phi = sum_i h_i on the tile + 3 ring (Eq. mac)
//   pass 2  grad phi, lap phi (Eqs. ICS-1st, ICS-sec), mu (Eq.
//           chemical_potential) and the form's level-1 fields on tile + 2
//   pass 3  interfacial + gravity force (Sec. 2.2), rho, u and phi u on
//           tile + 1 (Eq. mac)
//   pass 4  on the tile: P, div(phi u), d_t(phi u), BGK collision of f and h
//           with F_i and H_i (Eqs. fh, P_LBM, CH_LB_force), store of the
//           post-collision populations; streaming is the next step's pull.
// HBM traffic per node and step is the algorithmic state: 18 populations read
// and written plus (phi u) read and written; halo re-reads hit L1/L2.
//
// Two ways to obtain the pulled populations (StageMode, chosen per domain by
// the autotuner):
//   kBoxes   one 2-D box per population plane is staged in shared memory:
//            h planes on the tile + 3 ring, f planes on the tile + 1 ring,
//            each shifted by -c_i in y so that its rows hold pulled values; in
//            x all boxes span the same 16-byte aligned columns and the -c_ix
//            shift is applied on read.  Interior tiles issue the 18 boxes as
//            TMA tensor loads (cp.async.bulk.tensor) on an mbarrier, seam and
//            wall tiles fill them with cp.async; persistent CTAs walk tiles.
//   kGather  every pulled value is an L1-cached load from the population
//            planes; one CTA per tile.
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
// TMA, cp.async and mbarrier (inline PTX)
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
// 4-byte asynchronous copy global -> shared, zero-filled when !valid
__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_addr(dst)), "l"(src),
               "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}
// 16-byte asynchronous copy global -> shared, bypassing L1; zero-filled when
// !valid (nothing is read then)
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_addr(dst)), "l"(src),
               "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}

__host__ __device__ constexpr int pad128(int b) { return (b + 127) / 128 * 128; }

// ---------------------------------------------------------------------------
// shared-memory geometry: per-tile fields, and the box set of kBoxes
// ---------------------------------------------------------------------------
// TY: rows of the tile (kTY, or fewer for the batch's short tiles)
template <int FORM, bool TAPE = false, int TY = kTY>
struct Fields {
  static constexpr int B3X = kTX + 6, B3Y = TY + 6;  // tile + 3 ring
  static constexpr int B2X = kTX + 4, B2Y = TY + 4;  // tile + 2 ring
  static constexpr int B1X = kTX + 2, B1Y = TY + 2;  // tile + 1 ring
  static constexpr int N3 = B3X * B3Y, N2 = B2X * B2Y, N1 = B1X * B1Y;
  static constexpr int NE = extra_fields<FORM>();
  // lap phi is kept past pass 2 only by the forms whose force uses it (and
  // by the taping step, which records it)
  static constexpr bool kLap = FORM == kPF1 || FORM == kPF2 || TAPE;
  static constexpr int NS2 = 3 + (kLap ? 1 : 0) + NE;  // grad phi, mu, [lap], extras
  static constexpr int OFF_PHI = 0;
  static constexpr int OFF_S2 = OFF_PHI + pad128(N3 * 4);
  static constexpr int OFF_S1 = OFF_S2 + pad128(NS2 * N2 * 4);
  static constexpr int BYTES = OFF_S1 + pad128(6 * N1 * 4);
};

template <class ST>
struct Boxes {
  using T = typename ST::T;
  static constexpr int EB = sizeof(T);
  static constexpr int XPAD = box_xpad(EB);
  static constexpr int PW = box_w(EB);
  static constexpr int RH = kBoxRowsH, RF = kBoxRowsF;
  // h planes (h_0 in float32 when the storage is split), then f planes
  static constexpr int HB0 = pad128(RH * PW * (ST::kSplitH0 ? 4 : EB));
  static constexpr int HB = pad128(RH * PW * EB);
  static constexpr int FB = pad128(RF * PW * EB);
  static constexpr int BYTES = HB0 + 8 * HB + 9 * FB;
  static constexpr int TMA_TX = RH * PW * (ST::kSplitH0 ? 4 : EB) + 8 * RH * PW * EB +
                                9 * RF * PW * EB;  // bytes the 18 loads deliver
  __device__ static int h_off(int i) { return i == 0 ? 0 : HB0 + (i - 1) * HB; }
  __device__ static int f_off(int i) { return HB0 + 8 * HB + i * FB; }
};

// ---------------------------------------------------------------------------
// sources of pulled populations
// ---------------------------------------------------------------------------
// From the shared-memory box set bx.  Ring-3 node (r, cc) of pass 1, ring-1
// node (ly, lx) of pass 3 and tile node (ly, lx) of pass 4; the population i
// pulled at a node sits at box column (node column - c_ix) of its row.
template <class ST>
struct BoxSrc {
  static constexpr bool kInner = false, kWallX = false;
  using G = Boxes<ST>;
  const unsigned char* bx;
  // populations in the storage scale of the format
  template <int I>
  __device__ __forceinline__ float h(int r, int c, const Phys&) const {
    if constexpr (ST::kSplitH0 && I == 0) {
      return reinterpret_cast<const float*>(bx + G::h_off(0))[r * G::PW + c];
    } else {
      return ST::raw(reinterpret_cast<const typename ST::T*>(bx + G::h_off(I))[r * G::PW + c]);
    }
  }
  template <int I>
  __device__ __forceinline__ float f(int r, int c, const Phys&) const {
    return ST::raw(reinterpret_cast<const typename ST::T*>(bx + G::f_off(I))[r * G::PW + c]);
  }
  __device__ __forceinline__ float phi(const StepArgs& a, int r, int cc, int, int) const {
    const int c = cc + G::XPAD - 3;
    const Phys& P = a.p;
    float hh[9];
    hh[0] = h<0>(r, c, P);
    hh[1] = h<1>(r, c - 1, P);
    hh[2] = h<2>(r, c, P);
    hh[3] = h<3>(r, c + 1, P);
    hh[4] = h<4>(r, c, P);
    hh[5] = h<5>(r, c - 1, P);
    hh[6] = h<6>(r, c + 1, P);
    hh[7] = h<7>(r, c + 1, P);
    hh[8] = h<8>(r, c - 1, P);
    return phi_sum<ST>(hh, P);
  }
  __device__ __forceinline__ void f_ring1(const StepArgs& a, int ly, int lx, int, int,
                                          float* f) const {
    const int c = lx + G::XPAD - 1;
    const Phys& P = a.p;
    f[1] = this->f<1>(ly, c - 1, P);
    f[2] = this->f<2>(ly, c, P);
    f[3] = this->f<3>(ly, c + 1, P);
    f[4] = this->f<4>(ly, c, P);
    f[5] = this->f<5>(ly, c - 1, P);
    f[6] = this->f<6>(ly, c + 1, P);
    f[7] = this->f<7>(ly, c + 1, P);
    f[8] = this->f<8>(ly, c - 1, P);
  }
  __device__ __forceinline__ void f_node(const StepArgs& a, int ly, int lx, int, int,
                                         float* f) const {
    const int c = lx + G::XPAD, r = ly + 1;
    const Phys& P = a.p;
    f[0] = this->f<0>(r, c, P);
    f[1] = this->f<1>(r, c - 1, P);
    f[2] = this->f<2>(r, c, P);
    f[3] = this->f<3>(r, c + 1, P);
    f[4] = this->f<4>(r, c, P);
    f[5] = this->f<5>(r, c - 1, P);
    f[6] = this->f<6>(r, c + 1, P);
    f[7] = this->f<7>(r, c + 1, P);
    f[8] = this->f<8>(r, c - 1, P);
  }
  __device__ __forceinline__ void h_node(const StepArgs& a, int ly, int lx, int, int,
                                         float* hh) const {
    const int c = lx + G::XPAD, r = ly + 3;
    const Phys& P = a.p;
    hh[0] = h<0>(r, c, P);
    hh[1] = h<1>(r, c - 1, P);
    hh[2] = h<2>(r, c, P);
    hh[3] = h<3>(r, c + 1, P);
    hh[4] = h<4>(r, c, P);
    hh[5] = h<5>(r, c - 1, P);
    hh[6] = h<6>(r, c + 1, P);
    hh[7] = h<7>(r, c + 1, P);
    hh[8] = h<8>(r, c - 1, P);
  }
};

// Straight from the population planes (global coordinates of the node).
// INNER: the tile and its 3-ring pull only from inside the domain, so node
// coordinates need no wrap or mirror and pulls no ghost row.
// XW: free-slip side walls (specular pulls at x = 0 and nx - 1).
template <class ST, bool INNER = false, bool XW = false>
struct GatherSrc {
  static constexpr bool kInner = INNER, kWallX = XW;
  __device__ __forceinline__ static Pull idx(const Lattice& L, int gx, int gy) {
    if constexpr (INNER) return pull_idx_inner(L, gx, gy);
    else return pull_idx<XW>(L, gx, gy);
  }
  // populations in the storage scale of the format
  __device__ __forceinline__ float phi(const StepArgs& a, int, int, int gx, int gy) const {
    return pull_phi_s<ST>(a, idx(a.L, gx, gy));
  }
  __device__ __forceinline__ void f_ring1(const StepArgs& a, int, int, int gx, int gy,
                                          float* f) const {
    const Pull q = idx(a.L, gx, gy);
    f[1] = load_fs<ST, 1>(a, q.i[1]);
    f[2] = load_fs<ST, 2>(a, q.i[2]);
    f[3] = load_fs<ST, 3>(a, q.i[3]);
    f[4] = load_fs<ST, 4>(a, q.i[4]);
    f[5] = load_fs<ST, 5>(a, q.i[5]);
    f[6] = load_fs<ST, 6>(a, q.i[6]);
    f[7] = load_fs<ST, 7>(a, q.i[7]);
    f[8] = load_fs<ST, 8>(a, q.i[8]);
  }
  __device__ __forceinline__ void f_node(const StepArgs& a, int, int, int gx, int gy,
                                         float* f) const {
    pull_fs<ST>(a, idx(a.L, gx, gy), f);
  }
  __device__ __forceinline__ void h_node(const StepArgs& a, int, int, int gx, int gy,
                                         float* h) const {
    pull_hs<ST>(a, idx(a.L, gx, gy), h);
  }
};

// ---------------------------------------------------------------------------
// box staging
// ---------------------------------------------------------------------------
// Tiles (of TY rows) whose 3-ring and its pull sources lie inside the domain.
template <int TY = kTY>
__device__ __forceinline__ bool inner_tile(const Lattice& L, int x0, int y0) {
  return x0 >= 4 && x0 + kTX + 4 <= L.nx && y0 >= 4 && y0 + TY + 4 <= L.ny;
}

// Tiles whose 18 boxes lie inside the stored planes without wrapping.
template <class ST>
__device__ __forceinline__ bool tma_tile(const StepArgs& a, int x0, int y0) {
  using G = Boxes<ST>;
  return a.use_tma && x0 - G::XPAD >= 0 && x0 + kTX + G::XPAD <= a.L.nx && y0 >= 4 &&
         y0 + kTY + 4 <= a.L.ny;
}

// Issue the 18 box loads of the tile at (x0, y0) into box set bx (one thread).
// The tensor maps of `a` must live in parameter or global memory.
template <class ST>
__device__ __forceinline__ void issue_tma(const StepArgs& a, unsigned char* bx, uint64_t* bar,
                                          int x0, int y0) {
  using G = Boxes<ST>;
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

// storage row of source domain row yy, or -1 beyond a wall's ghost row
__device__ __forceinline__ int source_row(const Lattice& L, int yy) {
  if (L.wall) return (yy >= -1 && yy <= L.ny) ? yy + 1 : -1;
  return wrap(yy, L.ny) + 1;
}

// Fill the boxes of a seam or wall tile.  Box row r of plane i holds storage
// row (node row - c_iy) + 1 of the rows the tile needs; rows the tile never
// pulls (beyond a wall) are zero.  ASYNC (4-byte storage): cp.async per
// element, completed by cp_async_wait_all() and a CTA barrier; otherwise
// plain loads and stores.
template <class ST, int NT, bool ASYNC>
__device__ void fill_boxes(const StepArgs& a, unsigned char* bx, int x0, int y0) {
  using G = Boxes<ST>;
  using T = typename ST::T;
  const Lattice& L = a.L;
  for (int e = threadIdx.x; e < G::RH * G::PW; e += NT) {
    const int r = e / G::PW, c = e - r * G::PW;
    const int gx = wrap(x0 - G::XPAD + c, L.nx);
    const int yn = y0 - 3 + r;  // node row
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int sr = source_row(L, yn - qcy(i));
      const int off = sr >= 0 ? sr * L.nx + gx : 0;
      if (ST::kSplitH0 && i == 0) {
        float* d = reinterpret_cast<float*>(bx + G::h_off(0)) + e;
        *d = sr >= 0 ? a.h0_in[off] : 0.0f;
      } else {
        const int pl = ST::kSplitH0 ? i - 1 : i;
        const T* src = reinterpret_cast<const T*>(a.h_in) + (size_t)pl * L.plane + off;
        T* d = reinterpret_cast<T*>(bx + G::h_off(i)) + e;
        if constexpr (ASYNC) cp_async4(d, src, sr >= 0);
        else *d = sr >= 0 ? *src : T(0.0f);
      }
    }
  }
  for (int e = threadIdx.x; e < G::RF * G::PW; e += NT) {
    const int r = e / G::PW, c = e - r * G::PW;
    const int gx = wrap(x0 - G::XPAD + c, L.nx);
    const int yn = y0 - 1 + r;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int sr = source_row(L, yn - qcy(i));
      const T* src = reinterpret_cast<const T*>(a.f_in) + (size_t)i * L.plane +
                     (sr >= 0 ? sr * L.nx + gx : 0);
      T* d = reinterpret_cast<T*>(bx + G::f_off(i)) + e;
      if constexpr (ASYNC) cp_async4(d, src, sr >= 0);
      else *d = sr >= 0 ? *src : T(0.0f);
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

// ---------------------------------------------------------------------------
// collision of an opposite pair (i, j) with c_j = -c_i, w_j = w_i:
// f_i^+ = f_i (1 - 1/tau_f) + f_i^eq / tau_f + (1 - 1/(2 tau_f)) F_i and the
// same for h with tau_h and H_i (Eqs. fh, P_LBM, CH_LB_force, heq_CH).
// With s_i = 3 c_i.u + 4.5 (c_i.u)^2 - 1.5 |u|^2, a_i = c_i.F - u.F and
// b_i = a_i + c_i.R - u.R (R = grad rho / 3), the f update is
//   f_i^+ = (1 - omf) f_i + w omf P + w cff a_i + s_i (w omf rho/3 + w cff b_i)
// and the h update, with d_i = c_i.(d/dt)(phi u),
//   h_i^+ = (1 - omh) h_i + w (omh eta mu + chh A) + (c_i.u) w omh 3 phi
//           + d_i 3 w chh,
// so the weight enters through per-node constants of its class (axis or
// diagonal) and the pair shares c_i.u and d_i with opposite signs.
// ---------------------------------------------------------------------------
struct CollideConsts {
  float ux, uy, Fx, Fy, rx, ry, uF, uR, uu15, omf1, omh1, dtx, dty;
  float t1[2];  // w omf P
  float t2[2];  // w omf rho / 3
  float t3[2];  // w (1 - omf / 2)
  float hc[2];  // w (omh eta mu + chh A)
  float hu[2];  // 3 w omh phi
  float hd[2];  // 3 w chh
};
template <int I>
__device__ __forceinline__ void collide_pair(const CollideConsts& k, float fi, float fj, float hi,
                                             float hj, float& foi, float& foj, float& hoi,
                                             float& hoj) {
  constexpr int C = I <= 4 ? 0 : 1;
  constexpr float cx = (float)qcx(I), cy = (float)qcy(I);
  const float cu = cx * k.ux + cy * k.uy;
  const float q = (4.5f * cu) * cu - k.uu15;
  const float l = 3.0f * cu;
  const float si = q + l, sj = q - l;
  const float cF = cx * k.Fx + cy * k.Fy;
  const float cR = cx * k.rx + cy * k.ry;
  const float ai = cF - k.uF, aj = -cF - k.uF;
  const float bi = ai + (cR - k.uR), bj = aj - (cR + k.uR);
  foi = fmaf(k.omf1, fi, fmaf(si, fmaf(k.t3[C], bi, k.t2[C]), fmaf(k.t3[C], ai, k.t1[C])));
  foj = fmaf(k.omf1, fj, fmaf(sj, fmaf(k.t3[C], bj, k.t2[C]), fmaf(k.t3[C], aj, k.t1[C])));
  const float cd = cx * k.dtx + cy * k.dty;
  const float x = fmaf(cu, k.hu[C], cd * k.hd[C]);
  hoi = fmaf(k.omh1, hi, k.hc[C] + x);
  hoj = fmaf(k.omh1, hj, k.hc[C] - x);
}

// ---------------------------------------------------------------------------
// one tile: passes 1-4, populations from SRC, fields in shared memory fs
// ---------------------------------------------------------------------------
// TAPE: also record, per interior node, the step's intermediates that the
// adjoint reads (plane layout of the TapePlane enum, a.tape + plane * nx ny).
// OWN (one collision node per thread only): keep the own node's populations
// in registers between the passes (below).
// NEXT (two collision nodes per thread): issue the second node's pulls before
// the first node's collision (off where the extra live values would spill).
template <int FORM, class ST, int NT, class SRC, bool TAPE = false, int TY = kTY,
          bool OWN = kTX * TY == NT, bool NEXT = true>
__device__ __forceinline__ void step_tile(const StepArgs& a, const SRC& src, unsigned char* fs,
                                          int x0, int y0) {
  using F = Fields<FORM, TAPE, TY>;
  constexpr int B3X = F::B3X, B2X = F::B2X, B1X = F::B1X, B1Y = F::B1Y;
  constexpr int N2 = F::N2, N1 = F::N1;
  constexpr int NPT = kTX * TY / NT;  // collision nodes per thread
  static_assert(kTX * TY % NT == 0, "whole collision nodes per thread");
  // One collision node per thread (kOwn): the thread pulls its own node
  // first in passes 1 and 3 and keeps those populations, and the node's
  // force and velocity, in registers for pass 4, which then reads no plane;
  // the ring nodes follow.  Same arithmetic per node as the row-major order.
  static_assert(!OWN || NPT == 1, "own-node order needs one collision node per thread");
  constexpr bool kOwn = OWN;
  constexpr int NTILE = kTX * TY;
  // level-1 field slots in s2, ring-1 slots in s1
  constexpr int GX = 0, GY = 1, MU = 2, LAP = 3, E0 = F::kLap ? 4 : 3;
  constexpr int FX = 0, FY = 1, UX = 2, UY = 3, PUX = 4, PUY = 5;
  float* sPhi = reinterpret_cast<float*>(fs + F::OFF_PHI);
  float* s2 = reinterpret_cast<float*>(fs + F::OFF_S2);
  float* s1 = reinterpret_cast<float*>(fs + F::OFF_S1);
  const Lattice& L = a.L;
  const Phys& P = a.p;
  const int tid = threadIdx.x;
  const int nn = L.nx * L.ny;
  constexpr bool kIn = SRC::kInner;
  constexpr bool kXw = SRC::kWallX;  // free-slip side walls (mirror columns)
  // 16-bit formats: populations stay in their storage scale p_i 2^s / w_i
  // (h_0 excepted); moments and collision constants carry the weights
  constexpr bool kScaled = ST::kSplitH0;
  const auto col = [&](int x) { return kXw ? map_col(x, L.nx, 1) : wrap(x, L.nx); };

  // (phi u)^{t-1} of this thread's collision nodes, loaded first so that the
  // load latency overlaps passes 1-3
  float pu_prev_x[NPT], pu_prev_y[NPT];
#pragma unroll
  for (int j = 0; j < NPT; ++j) {
    const int k = tid + j * NT;
    const int gx = x0 + k % kTX, gy = y0 + k / kTX;
    pu_prev_x[j] = 0.0f;
    pu_prev_y[j] = 0.0f;
    if (!a.first && !a.macro && (kIn || (gx < L.nx && gy < L.ny))) {
      pu_prev_x[j] = a.phiu[gy * L.nx + gx];
      pu_prev_y[j] = a.phiu[nn + gy * L.nx + gx];
    }
  }

  // ---- pass 1: phi on tile + 3 ------------------------------------------------
  const auto phi_node = [&](int r, int cc) {
    const int yn = y0 - 3 + r;
    if (!kIn && L.wall && (yn < 0 || yn >= L.ny)) return;  // mirrored below
    sPhi[r * B3X + cc] = kIn ? src.phi(a, r, cc, x0 - 3 + cc, yn)
                             : src.phi(a, r, cc, col(x0 - 3 + cc), L.wall ? yn : wrap(yn, L.ny));
  };
  // own node of the thread (kOwn): tile node (oly, olx)
  const int oly = tid / kTX, olx = tid - oly * kTX;
  const int ogx = x0 + olx, ogy = y0 + oly;
  float hown[kOwn ? 9 : 1];
  if constexpr (kOwn) {
    if (kIn || !L.wall || ogy < L.ny) {
      if constexpr (kIn) src.h_node(a, oly, olx, ogx, ogy, hown);
      else src.h_node(a, oly, olx, col(ogx), L.wall ? ogy : wrap(ogy, L.ny), hown);
      sPhi[(oly + 3) * B3X + olx + 3] = phi_sum<ST>(hown, P);
    }
    // the 3-ring: 3 rows above and below, then 3 columns left and right
    const auto ring3 = [&](int m, int& r, int& cc) {
      if (m < 6 * B3X) {
        const int rr = m / B3X;
        r = rr < 3 ? rr : rr + TY;
        cc = m - rr * B3X;
      } else {
        const int q = (m - 6 * B3X) / 6, c6 = m - 6 * B3X - q * 6;
        r = 3 + q;
        cc = c6 < 3 ? c6 : kTX + c6;
      }
    };
    constexpr int R3 = F::N3 - NTILE;
    if constexpr (kIn && R3 <= 2 * NT) {
      // at most two ring nodes per thread: both pulls are issued before
      // either sum, so that the CTA waits for one round of loads, not two
      const bool v1 = R3 >= NT || tid < R3, v2 = tid + NT < R3;
      int r1, c1, r2, c2;
      ring3(v1 ? tid : 0, r1, c1);
      ring3(v2 ? tid + NT : 0, r2, c2);
      float p1 = 0.0f, p2 = 0.0f;
      if (v1) p1 = src.phi(a, r1, c1, x0 - 3 + c1, y0 - 3 + r1);
      if (v2) p2 = src.phi(a, r2, c2, x0 - 3 + c2, y0 - 3 + r2);
      if (v1) sPhi[r1 * B3X + c1] = p1;
      if (v2) sPhi[r2 * B3X + c2] = p2;
    } else {
      for (int m = tid; m < R3; m += NT) {
        int r, cc;
        ring3(m, r, cc);
        phi_node(r, cc);
      }
    }
  } else {
#pragma unroll 3
    for (int k = tid; k < F::N3; k += NT) {
      const int r = k / B3X;
      phi_node(r, k - r * B3X);
    }
  }
  __syncthreads();
  if (!kIn && L.wall && (y0 - 3 < 0 || y0 + TY + 3 > L.ny)) {
    // mirror ghosts of phi about the wall planes
    for (int k = tid; k < F::N3; k += NT) {
      const int r = k / B3X, cc = k - r * B3X;
      const int yn = y0 - 3 + r;
      if (yn >= 0 && yn < L.ny) continue;
      const int rm = map_row(yn, L.ny, 1) - (y0 - 3);
      sPhi[k] = (rm >= 0 && rm < F::B3Y) ? sPhi[rm * B3X + cc] : 0.0f;
    }
    __syncthreads();
  }

  // Float32 planes: f of this thread's first ring-1 node is loaded before
  // pass 2 so that a gather's latency overlaps it (16-bit planes, and the
  // STF-2 force's extra stencils, would spill the held values).  Box staging
  // takes the same order so that both modes round identically.
  // kOwn: the held values are the own node's f (all nine, for pass 4).
  constexpr bool kPre = sizeof(typename ST::T) == 4 && FORM != kSTF2;
  float fpre[9];
  const auto load_own_f = [&](float* f) {
    if constexpr (kIn) src.f_node(a, oly, olx, ogx, ogy, f);
    else src.f_node(a, oly, olx, col(ogx), map_row(ogy, L.ny, L.wall), f);
  };
  // kOwn on an inner tile: f of the thread's 1-ring node too (the threads
  // that have one), so that pass 3 waits for no load
  constexpr int R1 = F::N1 - NTILE;
  constexpr bool kPreRing = kPre && kOwn && kIn && R1 <= NT;
  const auto ring1 = [&](int m, int& ly1, int& lx1) {
    if (m < 2 * B1X) {
      ly1 = m < B1X ? 0 : TY + 1;
      lx1 = m < B1X ? m : m - B1X;
    } else {
      const int q = m - 2 * B1X;
      ly1 = 1 + (q >> 1);
      lx1 = (q & 1) ? kTX + 1 : 0;
    }
  };
  float fring[kPreRing ? 9 : 1];
  if constexpr (kPre && kOwn) {
    load_own_f(fpre);
    if constexpr (kPreRing) {
      if (tid < R1) {
        int ly1, lx1;
        ring1(tid, ly1, lx1);
        src.f_ring1(a, ly1, lx1, x0 - 1 + lx1, y0 - 1 + ly1, fring);
      }
    }
  } else if constexpr (kPre) {
    const int ly = tid / B1X, lx = tid - ly * B1X;
    if constexpr (kIn) src.f_ring1(a, ly, lx, x0 - 1 + lx, y0 - 1 + ly, fpre);
    else src.f_ring1(a, ly, lx, col(x0 - 1 + lx), map_row(y0 - 1 + ly, L.ny, L.wall), fpre);
  }

  // ---- pass 2: grad phi, lap phi, mu, level-1 fields on tile + 2 -------------
  for (int k = tid; k < N2; k += NT) {
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
    if constexpr (F::kLap) s2[LAP * N2 + k] = lap;
    s2[MU * N2 + k] = P.beta4 * pc * ((pc - 1.0f) * (pc + 1.0f)) - P.kappa * lap;
    if constexpr (FORM == kCSF1 || FORM == kCSF2) {
      const float inv = rsqrtf(gx * gx + gy * gy + P.eps2);
      s2[(E0 + 0) * N2 + k] = gx * inv;
      s2[(E0 + 1) * N2 + k] = gy * inv;
    }
  }
  __syncthreads();

  // ---- pass 3: force, rho, u, phi u on tile + 1 -----------------------------
  static_assert(N1 > NT, "every thread has a first ring-1 node");
  struct Node3 {
    float Fx, Fy, ux, uy;
  };
  auto pass3 = [&](int k, const float* f) -> Node3 {
    const int ly = k / B1X, lx = k - ly * B1X;
    const int c2 = (ly + 1) * B2X + lx + 1;
    const float phi = sPhi[(ly + 2) * B3X + lx + 2];
    const float gx = s2[GX * N2 + c2], gy = s2[GY * N2 + c2];
    float Fx, Fy;
    float a0 = 0.0f, a1 = 0.0f;  // what the force's adjoint needs (TapePlane TP_A0/1)
    if constexpr (FORM == kSTF1 || FORM == kSTF2) {
      // T = grad phi (x) grad phi, formed at each neighbour from the gradient
      const float* sgx = s2 + GX * N2;
      const float* sgy = s2 + GY * N2;
      const auto txx = [&](int i) { return sgx[i] * sgx[i]; };
      const auto txy = [&](int i) { return sgx[i] * sgy[i]; };
      const auto tyy = [&](int i) { return sgy[i] * sgy[i]; };
      Fx = -P.kappa * (ics_dx_of<B2X>(txx, c2) + ics_dy_of<B2X>(txy, c2));
      Fy = -P.kappa * (ics_dx_of<B2X>(txy, c2) + ics_dy_of<B2X>(tyy, c2));
      if constexpr (FORM == kSTF2) {
        // kappa grad |grad phi|^2 with |grad phi|^2 = Txx + Tyy at each node
        Fx += P.kappa * (ics_dx_of<B2X>(txx, c2) + ics_dx_of<B2X>(tyy, c2));
        Fy += P.kappa * (ics_dy_of<B2X>(txx, c2) + ics_dy_of<B2X>(tyy, c2));
      }
      a0 = Fx;
      a1 = Fy;
    } else if constexpr (FORM == kCPF1) {
      const float* mu = s2 + MU * N2;
      a0 = ics_dx<B2X>(mu, c2);
      a1 = ics_dy<B2X>(mu, c2);
      Fx = -phi * a0;
      Fy = -phi * a1;
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
      a0 = ics_dx<B2X>(lap, c2);
      a1 = ics_dy<B2X>(lap, c2);
      Fx = P.kappa * phi * a0;
      Fy = P.kappa * phi * a1;
    } else {  // CSF-1, CSF-2
      const float divn = ics_dx<B2X>(s2 + E0 * N2, c2) + ics_dy<B2X>(s2 + (E0 + 1) * N2, c2);
      a0 = divn;
      float coef;
      if constexpr (FORM == kCSF1) coef = -P.kappa * sqrtf(gx * gx + gy * gy) * divn;
      else coef = -P.half_sigma * divn;
      Fx = coef * gx;
      Fy = coef * gy;
    }
    const float rho = P.rho_mid + P.drho_half * phi;
    Fx += (rho - P.rho0) * P.gx;
    Fy += (rho - P.rho0) * P.gy;
    float jx, jy;
    f_flux<ST>(f, P, jx, jy);
    // Eq. mac: u = [sum c f + cs^2 F / 2] / (cs^2 rho)
    const float irho = __fdividef(1.0f, rho);
    const float ux = (3.0f * jx + 0.5f * Fx) * irho;
    const float uy = (3.0f * jy + 0.5f * Fy) * irho;
    if constexpr (!kOwn) {  // kOwn: pass 4 takes them from registers
      s1[FX * N1 + k] = Fx;
      s1[FY * N1 + k] = Fy;
    }
    s1[UX * N1 + k] = ux;
    s1[UY * N1 + k] = uy;
    s1[PUX * N1 + k] = phi * ux;
    s1[PUY * N1 + k] = phi * uy;
    if constexpr (TAPE) {
      const int gxn = x0 - 1 + lx, gyn = y0 - 1 + ly;
      if (lx >= 1 && lx <= kTX && ly >= 1 && ly <= TY && gxn < L.nx && gyn < L.ny) {
        float* t = a.tape + gyn * L.nx + gxn;
        t[TP_A0 * nn] = a0;
        t[TP_A1 * nn] = a1;
        t[TP_FX * nn] = Fx;
        t[TP_FY * nn] = Fy;
        t[TP_UX * nn] = ux;
        t[TP_UY * nn] = uy;
      }
    }
    return Node3{Fx, Fy, ux, uy};
  };
  auto load_ring1 = [&](int k, float* f) {
    const int ly = k / B1X, lx = k - ly * B1X;
    if constexpr (kIn) src.f_ring1(a, ly, lx, x0 - 1 + lx, y0 - 1 + ly, f);
    else src.f_ring1(a, ly, lx, col(x0 - 1 + lx), map_row(y0 - 1 + ly, L.ny, L.wall), f);
  };
  Node3 own3{};
  if constexpr (kOwn) {
    if constexpr (!kPre) load_own_f(fpre);
    own3 = pass3((oly + 1) * B1X + olx + 1, fpre);
    // the 1-ring: the rows above and below, then the columns left and right
    if constexpr (kPreRing) {
      if (tid < R1) {
        int ly1, lx1;
        ring1(tid, ly1, lx1);
        pass3(ly1 * B1X + lx1, fring);
      }
    } else {
      for (int m = tid; m < R1; m += NT) {
        int ly1, lx1;
        ring1(m, ly1, lx1);
        float f[9];
        load_ring1(ly1 * B1X + lx1, f);
        pass3(ly1 * B1X + lx1, f);
      }
    }
  } else {
    if constexpr (kPre) pass3(tid, fpre);
#pragma unroll 2
    for (int k = kPre ? tid + NT : tid; k < N1; k += NT) {
      float f[9];
      load_ring1(k, f);
      pass3(k, f);
    }
  }
  __syncthreads();

  // wall ghosts of phi u: phi (2 u_w - u) of the mirrored node
  if (!kIn && L.wall) {
    const int lb = -1 - (y0 - 1);      // ring-1 row of y = -1
    const int lt = L.ny - (y0 - 1);    // ring-1 row of y = ny
    const bool bot = lb >= 0 && lb + 1 < B1Y;
    const bool top = lt - 1 >= 0 && lt < B1Y;
    if (bot || top) {
      for (int lx = tid; lx < B1X; lx += NT) {
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
  // free-slip side walls: the ghost column of phi u is (-phi u_x, phi u_y) of
  // the mirrored column (after the y ghosts, so that the corners mirror them)
  if constexpr (kXw) {
    const int cl = -x0;             // ring-1 column of x = -1
    const int cr = L.nx - (x0 - 1);  // ring-1 column of x = nx
    const bool left = cl >= 0 && cl + 1 < B1X;
    const bool right = cr - 1 >= 0 && cr < B1X;
    if (left || right) {
      for (int ly = tid; ly < B1Y; ly += NT) {
        if (left) {
          const int g = ly * B1X + cl;
          s1[PUX * N1 + g] = -s1[PUX * N1 + g + 1];
          s1[PUY * N1 + g] = s1[PUY * N1 + g + 1];
        }
        if (right) {
          const int g = ly * B1X + cr;
          s1[PUX * N1 + g] = -s1[PUX * N1 + g - 1];
          s1[PUY * N1 + g] = s1[PUY * N1 + g - 1];
        }
      }
    }
    __syncthreads();
  }

  // ---- pass 4: collide and store on the tile --------------------------------
  // two collision nodes per thread on an inner tile: the second node's pulls
  // are issued before the first node's collision, so that they arrive while
  // it runs (measured faster for STF-1, CPF and PF; the STF-2 and CSF forces
  // then spill, and run slower)
  constexpr bool kNext = NEXT && !kOwn && NPT == 2 && kIn && FORM != kSTF2 && FORM != kCSF1 &&
                         FORM != kCSF2;
  float fnx[kNext ? 9 : 1], hnx[kNext ? 9 : 1];
  if constexpr (kNext) {
    const int k1 = tid + NT, ly1 = k1 / kTX, lx1 = k1 - ly1 * kTX;
    src.f_node(a, ly1, lx1, x0 + lx1, y0 + ly1, fnx);
    src.h_node(a, ly1, lx1, x0 + lx1, y0 + ly1, hnx);
  }
#pragma unroll
  for (int j = 0; j < NPT; ++j) {
    const int k = tid + j * NT;
    const int ly = k / kTX, lx = k - ly * kTX;
    const int gx = x0 + lx, gy = y0 + ly;
    if (!kIn && (gx >= L.nx || gy >= L.ny)) continue;
    const int c1 = (ly + 1) * B1X + lx + 1;
    const int c2 = (ly + 2) * B2X + lx + 2;
    const float phi = sPhi[(ly + 3) * B3X + lx + 3];
    const float Gx = s2[GX * N2 + c2], Gy = s2[GY * N2 + c2];
    const float mu = s2[MU * N2 + c2];
    const float Fx = kOwn ? own3.Fx : s1[FX * N1 + c1];
    const float Fy = kOwn ? own3.Fy : s1[FY * N1 + c1];
    const float ux = kOwn ? own3.ux : s1[UX * N1 + c1];
    const float uy = kOwn ? own3.uy : s1[UY * N1 + c1];
    const float rho = P.rho_mid + P.drho_half * phi;
    const float drx = P.drho_half * Gx, dry = P.drho_half * Gy;

    float f[9];
    if constexpr (kOwn) {
#pragma unroll
      for (int i = 0; i < 9; ++i) f[i] = fpre[i];
    } else if (kNext && j == 1) {
#pragma unroll
      for (int i = 0; i < 9; ++i) f[i] = fnx[kNext ? i : 0];
    } else {
      src.f_node(a, ly, lx, gx, gy, f);
    }
    const float sumf = f_sum<ST>(f, P);
    // Eq. mac: P = sum f + cs^2/2 u . grad rho
    const float Pr = sumf + (ux * drx + uy * dry) * (1.0f / 6.0f);
    // div(phi u) by Eq. ICS-1st on the ring-1 values
    const float div = ics_dx<B1X>(s1 + PUX * N1, c1) + ics_dy<B1X>(s1 + PUY * N1, c1);
    const int n_idx = gy * L.nx + gx;
    const float pux = phi * ux, puy = phi * uy;
    float dtx = 0.0f, dty = 0.0f;
    if (!a.first) {
      dtx = pux - pu_prev_x[j];
      dty = puy - pu_prev_y[j];
    }

    if (a.macro) {
      const float g2 = Gx * Gx + Gy * Gy;
      const float om = (1.0f - phi) * (1.0f + phi);
      const float f0e = 0.25f * P.beta4 * om * om;
      float ph = Pr;
      // p_h from the generalised pressure of the form (Eqs. SF2, P3456;
      // STF-1: P = p_h - kappa |grad phi|^2, the sign that Eqs. SF1, SF2
      // and P3456 imply together)
      if constexpr (FORM == kSTF1) ph = Pr + P.kappa * g2;
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
    if (!a.keep_phiu) {
      a.phiu[n_idx] = pux;
      a.phiu[nn + n_idx] = puy;
    }

    if constexpr (TAPE) {
      float* t = a.tape + n_idx;
#pragma unroll
      for (int i = 0; i < 9; ++i) t[(TP_F0 + i) * nn] = f[i];
      t[TP_PHI * nn] = phi;
      t[TP_GX * nn] = Gx;
      t[TP_GY * nn] = Gy;
      t[TP_L * nn] = s2[LAP * N2 + c2];
      t[TP_MU * nn] = mu;
      t[TP_PR * nn] = Pr;
      t[TP_DIV * nn] = div;
      t[TP_DTX * nn] = dtx;
      t[TP_DTY * nn] = dty;
    }

    float h[9];
    if constexpr (kOwn) {
#pragma unroll
      for (int i = 0; i < 9; ++i) h[i] = hown[i];
    } else if (kNext && j == 1) {
#pragma unroll
      for (int i = 0; i < 9; ++i) h[i] = hnx[kNext ? i : 0];
    } else {
      src.h_node(a, ly, lx, gx, gy, h);
    }

    // relaxation: tau_f = 1/2 + mu(phi) / (cs^2 rho) (Sec. 3)
    const float mv = P.mu_mid + P.mu_dhalf * phi;
    const float omf = __fdividef(1.0f, 0.5f + 3.0f * mv * __fdividef(1.0f, rho));
    const float cff = 1.0f - 0.5f * omf;
    const float emu = P.eta * mu;
    const float A = P.acoef * div;
    CollideConsts K;
    K.ux = ux;
    K.uy = uy;
    K.Fx = Fx;
    K.Fy = Fy;
    K.rx = drx * (1.0f / 3.0f);
    K.ry = dry * (1.0f / 3.0f);
    K.uF = ux * Fx + uy * Fy;
    K.uR = ux * K.rx + uy * K.ry;
    K.uu15 = 1.5f * (ux * ux + uy * uy);
    K.omf1 = 1.0f - omf;
    K.omh1 = 1.0f - P.inv_tau_h;
    K.dtx = dtx;
    K.dty = dty;
    {
      const float oP = omf * Pr, oR = omf * rho * (1.0f / 3.0f);
      const float hb = fmaf(P.inv_tau_h, emu, P.hforce * A);
      const float hp = 3.0f * P.inv_tau_h * phi, hd = 3.0f * P.hforce;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        // weight of the class (float32), or the storage scale 2^s, which
        // replaces w / w in the 16-bit scale p_i 2^s / w_i
        constexpr float wa = qw(1), wd = qw(5);
        const float wf = kScaled ? P.sf : (c == 0 ? wa : wd);
        const float wh = kScaled ? P.sh : (c == 0 ? wa : wd);
        K.t1[c] = wf * oP;
        K.t2[c] = wf * oR;
        K.t3[c] = wf * cff;
        K.hc[c] = wh * hb;
        K.hu[c] = wh * hp;
        K.hd[c] = wh * hd;
      }
    }

    float fo[9], ho[9];
    {
      // rest population: s_0 = -1.5 |u|^2, c_0 = 0, wbar_0 = w_0 - 1
      constexpr float w0 = qw(0);
      const float wf0 = kScaled ? P.sf : w0;
      const float s0 = -K.uu15;
      const float a0 = -K.uF, b0 = -K.uF - K.uR;
      fo[0] = fmaf(K.omf1, f[0],
                   wf0 * (fmaf(omf, Pr, cff * a0) + s0 * fmaf(omf, rho * (1.0f / 3.0f), cff * b0)));
      const float heq0 = phi + (w0 - 1.0f) * emu;
      ho[0] = fmaf(K.omh1, h[0], fmaf(P.inv_tau_h, heq0, P.hforce * ((w0 - 1.0f) * A)));
    }
    collide_pair<1>(K, f[1], f[3], h[1], h[3], fo[1], fo[3], ho[1], ho[3]);
    collide_pair<2>(K, f[2], f[4], h[2], h[4], fo[2], fo[4], ho[2], ho[4]);
    collide_pair<5>(K, f[5], f[7], h[5], h[7], fo[5], fo[7], ho[5], ho[7]);
    collide_pair<6>(K, f[6], f[8], h[6], h[8], fo[6], fo[8], ho[6], ho[8]);

    const int o = (gy + 1) * L.nx + gx;
    store_fs<ST, 0>(a, o, fo[0]); store_hs<ST, 0>(a, o, ho[0]);
    store_fs<ST, 1>(a, o, fo[1]); store_hs<ST, 1>(a, o, ho[1]);
    store_fs<ST, 2>(a, o, fo[2]); store_hs<ST, 2>(a, o, ho[2]);
    store_fs<ST, 3>(a, o, fo[3]); store_hs<ST, 3>(a, o, ho[3]);
    store_fs<ST, 4>(a, o, fo[4]); store_hs<ST, 4>(a, o, ho[4]);
    store_fs<ST, 5>(a, o, fo[5]); store_hs<ST, 5>(a, o, ho[5]);
    store_fs<ST, 6>(a, o, fo[6]); store_hs<ST, 6>(a, o, ho[6]);
    store_fs<ST, 7>(a, o, fo[7]); store_hs<ST, 7>(a, o, ho[7]);
    store_fs<ST, 8>(a, o, fo[8]); store_hs<ST, 8>(a, o, ho[8]);

    if (!kIn && L.wall) {
      // Ladd half-way bounce-back (Sec. 4): a population heading into the
      // wall returns to this node reversed, minus 2 w_i rho c_i.u_w (f) and
      // 2 w_i phi c_i.u_w / cs^2 (h); it is written into the ghost row the
      // next pull reads it from.
      const int xr = gx + 1 < L.nx ? gx + 1 : 0;        // x + 1
      const int xl = gx - 1 >= 0 ? gx - 1 : L.nx - 1;   // x - 1
      // beyond a free-slip side wall the ghost-row slot of x -+ 1 is the
      // mirror direction's slot in this column (where the specular pull reads)
      const bool lw = kXw && gx == 0, rw = kXw && gx == L.nx - 1;
      // diagonal weight w_5..8 (float32), or the storage scale in which
      // 2 w_i rho c_i.u_w / w_i is 2 rho c_i.u_w 2^s
      const float bwf = kScaled ? P.sf : qw(7), bwh = kScaled ? P.sh : qw(7);
      if (gy == 0) {
        const float uw = P.uwb;
        // i = 4 (0,-1) -> opp 2 at (x, -1); i = 7 (-1,-1) -> opp 5 at (x-1, -1);
        // i = 8 (1,-1) -> opp 6 at (x+1, -1)
        store_fs<ST, 2>(a, gx, fo[4]);
        store_hs<ST, 2>(a, gx, ho[4]);
        const float f5 = fo[7] - 2.0f * bwf * rho * (-uw);
        const float h5 = ho[7] - 2.0f * bwh * phi * 3.0f * (-uw);
        if (lw) {
          store_fs<ST, 6>(a, gx, f5);
          store_hs<ST, 6>(a, gx, h5);
        } else {
          store_fs<ST, 5>(a, xl, f5);
          store_hs<ST, 5>(a, xl, h5);
        }
        const float f6 = fo[8] - 2.0f * bwf * rho * uw;
        const float h6 = ho[8] - 2.0f * bwh * phi * 3.0f * uw;
        if (rw) {
          store_fs<ST, 5>(a, gx, f6);
          store_hs<ST, 5>(a, gx, h6);
        } else {
          store_fs<ST, 6>(a, xr, f6);
          store_hs<ST, 6>(a, xr, h6);
        }
      }
      if (gy == L.ny - 1) {
        const float uw = P.uwt;
        const int g = (L.ny + 1) * L.nx;
        // i = 2 (0,1) -> opp 4 at (x, ny); i = 5 (1,1) -> opp 7 at (x+1, ny);
        // i = 6 (-1,1) -> opp 8 at (x-1, ny)
        store_fs<ST, 4>(a, g + gx, fo[2]);
        store_hs<ST, 4>(a, g + gx, ho[2]);
        const float f7 = fo[5] - 2.0f * bwf * rho * uw;
        const float h7 = ho[5] - 2.0f * bwh * phi * 3.0f * uw;
        if (rw) {
          store_fs<ST, 8>(a, g + gx, f7);
          store_hs<ST, 8>(a, g + gx, h7);
        } else {
          store_fs<ST, 7>(a, g + xr, f7);
          store_hs<ST, 7>(a, g + xr, h7);
        }
        const float f8 = fo[6] - 2.0f * bwf * rho * (-uw);
        const float h8 = ho[6] - 2.0f * bwh * phi * 3.0f * (-uw);
        if (lw) {
          store_fs<ST, 7>(a, g + gx, f8);
          store_hs<ST, 7>(a, g + gx, h8);
        } else {
          store_fs<ST, 8>(a, g + xl, f8);
          store_hs<ST, 8>(a, g + xl, h8);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
// kBoxes: persistent CTAs, each walking tiles t = blockIdx.x + k gridDim.x;
// the box set of the next tile is staged when the current one is done (two
// CTAs per SM overlap one another's staging and compute).
template <int FORM, class ST>
__global__ void __launch_bounds__(kThreadsBoxes, kBlocksBoxes)
    k_step_boxes(const __grid_constant__ StepArgs a) {
  using G = Boxes<ST>;
  constexpr int NT = kThreadsBoxes;
  constexpr bool kAsync = sizeof(typename ST::T) == 4;
  extern __shared__ __align__(128) unsigned char sm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm);
  unsigned char* bx = sm + 128;
  unsigned char* fs = bx + G::BYTES;

  const int ntx = (a.L.nx + kTX - 1) / kTX;
  const int ntiles = ntx * ((a.L.ny + kTY - 1) / kTY);
  int t = blockIdx.x;
  if (t >= ntiles) return;
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  uint32_t parity = 0u;
  const BoxSrc<ST> src{bx};
  for (; t < ntiles; t += gridDim.x) {
    const int x0 = (t % ntx) * kTX, y0 = (t / ntx) * kTY;
    if (tma_tile<ST>(a, x0, y0)) {
      if (threadIdx.x == 0) issue_tma<ST>(a, bx, bar, x0, y0);
      if (!wait_boxes(a, bar, parity)) return;
      parity ^= 1u;
    } else {
      fill_boxes<ST, NT, kAsync>(a, bx, x0, y0);
      if constexpr (kAsync) cp_async_wait_all();
      __syncthreads();
    }
    step_tile<FORM, ST, NT>(a, src, fs, x0, y0);
    __syncthreads();
  }
}

// kGather: one CTA per tile, populations gathered through L1.  XW: free-slip
// side walls (a separate instantiation, so periodic domains run unchanged code).
// NT threads per 32 x TY tile, MINB CTAs per SM: kGather runs 32 x 16 tiles
// (two collision nodes per thread), kGather8 32 x 8 tiles (one, own-node
// order).
template <int FORM, class ST, bool XW, int NT, int TY, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_step_gather(const __grid_constant__ StepArgs a) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int ntx = (a.L.nx + kTX - 1) / kTX;
  const int x0 = (blockIdx.x % ntx) * kTX, y0 = (blockIdx.x / ntx) * TY;
  if (inner_tile<TY>(a.L, x0, y0))
    step_tile<FORM, ST, NT, GatherSrc<ST, true>, false, TY>(a, GatherSrc<ST, true>{}, sm, x0, y0);
  else
    step_tile<FORM, ST, NT, GatherSrc<ST, false, XW>, false, TY>(a, GatherSrc<ST, false, XW>{},
                                                                 sm, x0, y0);
}
template <int FORM, class ST, int NT, int TY, int MINB>
cudaError_t launch_gather(const StepArgs& a, cudaStream_t s, bool& configured) {
  constexpr int kBytes = Fields<FORM, false, TY>::BYTES;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_step_gather<FORM, ST, false, NT, TY, MINB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kBytes);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_step_gather<FORM, ST, true, NT, TY, MINB>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, kBytes);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int ntiles = ((a.L.nx + kTX - 1) / kTX) * ((a.L.ny + TY - 1) / TY);
  if (a.L.wall_x) k_step_gather<FORM, ST, true, NT, TY, MINB><<<ntiles, NT, kBytes, s>>>(a);
  else k_step_gather<FORM, ST, false, NT, TY, MINB><<<ntiles, NT, kBytes, s>>>(a);
  return cudaGetLastError();
}

// Taping step of the adjoint's recomputation (float32 storage, gathers): the
// plain step plus the record of its intermediates in a.tape.  Built for three
// CTAs per SM so that the extra live values do not spill.
template <int FORM>
__global__ void __launch_bounds__(kThreadsGather, 3) k_step_tape(const __grid_constant__ StepArgs a) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int ntx = (a.L.nx + kTX - 1) / kTX;
  const int x0 = (blockIdx.x % ntx) * kTX, y0 = (blockIdx.x / ntx) * kTY;
  if (inner_tile(a.L, x0, y0))
    step_tile<FORM, StoreF32, kThreadsGather, GatherSrc<StoreF32, true>, true>(
        a, GatherSrc<StoreF32, true>{}, sm, x0, y0);
  else
    step_tile<FORM, StoreF32, kThreadsGather, GatherSrc<StoreF32, false>, true>(
        a, GatherSrc<StoreF32, false>{}, sm, x0, y0);
}

int num_sms();

// the marching variant (march_kernel.cuh)
template <int FORM, class ST>
cudaError_t launch_march(const StepArgs& a, cudaStream_t s);

template <int FORM, class ST>
cudaError_t launch_form(int mode, const StepArgs& a, cudaStream_t s) {
  // the macroscopic read-back always takes the tile kernels
  if (mode == kMarch && !a.macro) return launch_march<FORM, ST>(a, s);
  static bool cfg[2] = {false, false};  // per instantiation and tile height
  if (mode == kGather8)
    return launch_gather<FORM, ST, kThreadsGather, kShortRows, kBlocksGather>(a, s, cfg[1]);
  if (mode != kBoxes)
    return launch_gather<FORM, ST, kThreadsGather, kTY, kBlocksGather>(a, s, cfg[0]);
  static bool configured = false;
  constexpr int kBoxBytes = 128 + Boxes<ST>::BYTES + Fields<FORM>::BYTES;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_step_boxes<FORM, ST>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, kBoxBytes);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int ntiles = ((a.L.nx + kTX - 1) / kTX) * ((a.L.ny + kTY - 1) / kTY);
  const int slots = num_sms() * kBlocksBoxes;
  k_step_boxes<FORM, ST><<<ntiles < slots ? ntiles : slots, kThreadsBoxes, kBoxBytes, s>>>(a);
  return cudaGetLastError();
}

template <class ST>
cudaError_t launch_step_impl(int form, int mode, const StepArgs& a, cudaStream_t s) {
  switch (form) {
    case kSTF1: return launch_form<kSTF1, ST>(mode, a, s);
    case kSTF2: return launch_form<kSTF2, ST>(mode, a, s);
    case kCPF1: return launch_form<kCPF1, ST>(mode, a, s);
    case kCPF2: return launch_form<kCPF2, ST>(mode, a, s);
    case kPF1: return launch_form<kPF1, ST>(mode, a, s);
    case kPF2: return launch_form<kPF2, ST>(mode, a, s);
    case kCSF1: return launch_form<kCSF1, ST>(mode, a, s);
    case kCSF2: return launch_form<kCSF2, ST>(mode, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pflbm

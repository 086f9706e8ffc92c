// Device helpers shared by the step kernel and the auxiliary kernels: the
// D2Q9 lattice (Sec. 3 of Zhang, Liang & Guo, arXiv 2012.14729), population
// storage formats, pull indexing with ghost rows for half-way bounce-back
// walls (Sec. 4), and the isotropic central-scheme stencils (Eqs. ICS-1st,
// ICS-sec) on shared-memory arrays.
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
  return (FORM == kCSF1 || FORM == kCSF2) ? 2 : 0;
}

// ---------------------------------------------------------------------------
// storage formats
// ---------------------------------------------------------------------------
// 16-bit formats store p_i 2^s / w_i (h_0 in float32).  dec/enc convert to
// and from the population value; raw/enc_raw only change the type, for the
// step kernel, which computes in that storage scale (the weights and 2^s then
// sit in its per-node constants).
struct StoreF32 {
  static constexpr bool kSplitH0 = false;
  using T = float;
  __device__ static __forceinline__ float dec(T v, float w_inv_scale) { return v; }
  __device__ static __forceinline__ T enc(float v, float scale_over_w) { return v; }
  __device__ static __forceinline__ float raw(T v) { return v; }
  __device__ static __forceinline__ T enc_raw(float v) { return v; }
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
  __device__ static __forceinline__ float raw(T v) { return __half2float(v); }
  __device__ static __forceinline__ T enc_raw(float v) { return __float2half_rn(v); }
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
  __device__ static __forceinline__ float raw(T v) { return __bfloat162float(v); }
  __device__ static __forceinline__ T enc_raw(float v) { return __float2bfloat16_rn(v); }
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

// The same in the storage scale of the format (the step kernel's arithmetic).
// The element offset of plane pl, index idx is formed in 32 bits (the host
// refuses lattices whose 9 planes reach 2^31 elements), so that one 32-bit
// add and one widening multiply-add address each population.
template <class ST, int I>
__device__ __forceinline__ float load_fs(const StepArgs& a, int idx) {
  using T = typename ST::T;
  return ST::raw(__ldg(reinterpret_cast<const T*>(a.f_in) + (unsigned)(I * a.L.plane + idx)));
}
template <class ST, int I>
__device__ __forceinline__ float load_hs(const StepArgs& a, int idx) {
  using T = typename ST::T;
  if constexpr (ST::kSplitH0 && I == 0) return __ldg(a.h0_in + (unsigned)idx);
  const int pl = ST::kSplitH0 ? I - 1 : I;
  return ST::raw(__ldg(reinterpret_cast<const T*>(a.h_in) + (unsigned)(pl * a.L.plane + idx)));
}
template <class ST, int I>
__device__ __forceinline__ void store_fs(const StepArgs& a, int idx, float v) {
  using T = typename ST::T;
  reinterpret_cast<T*>(a.f_out)[(unsigned)(I * a.L.plane + idx)] = ST::enc_raw(v);
}
template <class ST, int I>
__device__ __forceinline__ void store_hs(const StepArgs& a, int idx, float v) {
  using T = typename ST::T;
  if constexpr (ST::kSplitH0 && I == 0) {
    a.h0_out[(unsigned)idx] = v;
  } else {
    const int pl = ST::kSplitH0 ? I - 1 : I;
    reinterpret_cast<T*>(a.h_out)[(unsigned)(pl * a.L.plane + idx)] = ST::enc_raw(v);
  }
}

// Moments of populations in storage scale (h_0 and FP32 values as is):
// phi = sum h_i, sum f_i and j = sum c_i f_i.  FP32 sums in direction order;
// the 16-bit scale groups the directions of one weight class.
template <class ST>
__device__ __forceinline__ float phi_sum(const float* h, const Phys& P) {
  if constexpr (ST::kSplitH0) {
    const float ax = (h[1] + h[2]) + (h[3] + h[4]), dg = (h[5] + h[6]) + (h[7] + h[8]);
    return h[0] + fmaf(qw(1) * P.inv_sh, ax, (qw(5) * P.inv_sh) * dg);
  } else {
    float t = h[0];
    t += h[1];
    t += h[2];
    t += h[3];
    t += h[4];
    t += h[5];
    t += h[6];
    t += h[7];
    t += h[8];
    return t;
  }
}
template <class ST>
__device__ __forceinline__ float f_sum(const float* f, const Phys& P) {
  if constexpr (ST::kSplitH0) {
    const float ax = (f[1] + f[2]) + (f[3] + f[4]), dg = (f[5] + f[6]) + (f[7] + f[8]);
    return fmaf(qw(0) * P.inv_sf, f[0], fmaf(qw(1) * P.inv_sf, ax, (qw(5) * P.inv_sf) * dg));
  } else {
    return f[0] + (f[1] + f[2] + f[3] + f[4]) + (f[5] + f[6] + f[7] + f[8]);
  }
}
template <class ST>
__device__ __forceinline__ void f_flux(const float* f, const Phys& P, float& jx, float& jy) {
  if constexpr (ST::kSplitH0) {
    const float ca = qw(1) * P.inv_sf, cd = qw(5) * P.inv_sf;
    jx = fmaf(ca, f[1] - f[3], cd * ((f[5] - f[6]) + (f[8] - f[7])));
    jy = fmaf(ca, f[2] - f[4], cd * ((f[5] - f[8]) + (f[6] - f[7])));
  } else {
    jx = (f[1] - f[3]) + ((f[5] - f[6]) + (f[8] - f[7]));
    jy = (f[2] - f[4]) + ((f[5] - f[8]) + (f[6] - f[7]));
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

// Column of a scalar-field node: periodic wrap, or mirror about free-slip
// side walls (ghost column -k = column k - 1).
__device__ __forceinline__ int map_col(int x, int nx, int wall_x) {
  if (x >= 0 && x < nx) return x;
  if (!wall_x) return wrap(x, nx);
  while (x < 0 || x >= nx) x = (x < 0) ? -x - 1 : 2 * nx - 1 - x;
  return x;
}

// Storage indices of the 9 pulled populations of node (x, y), 0 <= x < nx,
// 0 <= y < ny: population i comes from (x - cx_i, y - cy_i); storage row is
// domain row + 1 (ghost rows 0 and ny + 1 hold bounced populations).  At a
// free-slip side wall a population whose source lies beyond the wall is the
// specular reflection of the population leaving the node's own column in the
// mirror direction (cx reversed): the index then points into that
// population's plane (planes are `plane` elements apart).
struct Pull {
  int i[9];
};
template <bool XW = false>
__device__ __forceinline__ Pull pull_idx(const Lattice& L, int x, int y) {
  int xm = x + 1, xp = x - 1;  // source columns for cx = -1 and cx = +1
  int dm = 0, dp = 0;          // plane offset (in planes) of the mirror direction
  if (xm >= L.nx) {
    if (XW) xm = x, dm = 1;  // 3 <- 1, 6 <- 5, 7 <- 8
    else xm -= L.nx;
  }
  if (xp < 0) {
    if (XW) xp = x, dp = 1;  // 1 <- 3, 5 <- 6, 8 <- 7
    else xp += L.nx;
  }
  int ym = y + 1, yp = y - 1;  // source rows for cy = -1 and cy = +1
  if (!L.wall) {
    if (ym >= L.ny) ym -= L.ny;
    if (yp < 0) yp += L.ny;
  }
  const int r0 = (y + 1) * L.nx, rm = (ym + 1) * L.nx, rp = (yp + 1) * L.nx;
  const int pl = L.plane;
  Pull p;
  p.i[0] = r0 + x;
  p.i[1] = r0 + xp + dp * 2 * pl;
  p.i[2] = rp + x;
  p.i[3] = r0 + xm - dm * 2 * pl;
  p.i[4] = rm + x;
  p.i[5] = rp + xp + dp * pl;
  p.i[6] = rp + xm - dm * pl;
  p.i[7] = rm + xm + dm * pl;
  p.i[8] = rm + xp - dp * pl;
  return p;
}

// The same for a node whose 8 neighbours lie inside the domain (no wrap, no
// ghost row): row and column offsets only.
__device__ __forceinline__ Pull pull_idx_inner(const Lattice& L, int x, int y) {
  const int r0 = (y + 1) * L.nx + x, rm = r0 + L.nx, rp = r0 - L.nx;
  Pull p;
  p.i[0] = r0;
  p.i[1] = r0 - 1;
  p.i[2] = rp;
  p.i[3] = r0 + 1;
  p.i[4] = rm;
  p.i[5] = rp - 1;
  p.i[6] = rp + 1;
  p.i[7] = rm + 1;
  p.i[8] = rm - 1;
  return p;
}

// pulled populations in storage scale, and phi from them
template <class ST>
__device__ __forceinline__ void pull_hs(const StepArgs& a, const Pull& q, float* h) {
  h[0] = load_hs<ST, 0>(a, q.i[0]);
  h[1] = load_hs<ST, 1>(a, q.i[1]);
  h[2] = load_hs<ST, 2>(a, q.i[2]);
  h[3] = load_hs<ST, 3>(a, q.i[3]);
  h[4] = load_hs<ST, 4>(a, q.i[4]);
  h[5] = load_hs<ST, 5>(a, q.i[5]);
  h[6] = load_hs<ST, 6>(a, q.i[6]);
  h[7] = load_hs<ST, 7>(a, q.i[7]);
  h[8] = load_hs<ST, 8>(a, q.i[8]);
}
template <class ST>
__device__ __forceinline__ void pull_fs(const StepArgs& a, const Pull& q, float* f) {
  f[0] = load_fs<ST, 0>(a, q.i[0]);
  f[1] = load_fs<ST, 1>(a, q.i[1]);
  f[2] = load_fs<ST, 2>(a, q.i[2]);
  f[3] = load_fs<ST, 3>(a, q.i[3]);
  f[4] = load_fs<ST, 4>(a, q.i[4]);
  f[5] = load_fs<ST, 5>(a, q.i[5]);
  f[6] = load_fs<ST, 6>(a, q.i[6]);
  f[7] = load_fs<ST, 7>(a, q.i[7]);
  f[8] = load_fs<ST, 8>(a, q.i[8]);
}
template <class ST>
__device__ __forceinline__ float pull_phi_s(const StepArgs& a, const Pull& q) {
  float h[9];
  pull_hs<ST>(a, q, h);
  return phi_sum<ST>(h, a.p);
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

// The same stencils of a field given as a function of the element index
// (products of stored fields formed at each neighbour).
template <int S, class Fn>
__device__ __forceinline__ float ics_dx_of(const Fn& a, int c) {
  return (a(c + 1) - a(c - 1)) * (1.0f / 3.0f) +
         ((a(c + S + 1) - a(c + S - 1)) + (a(c - S + 1) - a(c - S - 1))) * (1.0f / 12.0f);
}
template <int S, class Fn>
__device__ __forceinline__ float ics_dy_of(const Fn& a, int c) {
  return (a(c + S) - a(c - S)) * (1.0f / 3.0f) +
         ((a(c + S + 1) - a(c - S + 1)) + (a(c + S - 1) - a(c - S - 1))) * (1.0f / 12.0f);
}

}  // namespace pflbm

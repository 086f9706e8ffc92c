// Marching variant of the fused coupled step (Sec. 3 of Zhang, Liang & Guo,
// arXiv 2012.14729) for sm_103a: the same per-node arithmetic as step_tile
// in step_kernel.cuh, organised as a sweep along y instead of halo tiles.
//
// A persistent CTA owns contiguous runs of rows of a kMW-wide column strip
// and walks down them kMR rows per iteration.  Per iteration with output
// rows [y, y + kMR) its threads
//   - issue 16-byte cp.async copies of the population rows the next
//     iteration needs into a ring of row slots in shared memory: for every
//     node row, the 18 pulled population rows of the strip (each plane's row
//     shifted by -c_iy, the strip's columns plus a 16-byte aligned halo) and
//     the row of (phi u)^{t-1}.  Periodic seams are resolved chunk by chunk
//     and wall ghost rows are ordinary storage rows, so no stage below wraps
//     an index; the copies land while this iteration computes;
//   - run
//       A  phi = sum_i h_i                    on rows [y+3, y+kMR+3), strip+3
//       B  grad phi, lap phi, mu, form fields on rows [y+2, y+kMR+2), strip+2
//          (Eqs. ICS-1st, ICS-sec, chemical_potential)
//       C  force (Sec. 2.2) + gravity, rho, u, phi u (Eq. mac)
//                                             on rows [y+1, y+kMR+1), strip+1
//       D  P, div(phi u), d_t(phi u), collision of f and h and the store of
//          the post-collision populations (Eqs. fh, P_LBM, CH_LB_force)
//                                             on rows [y, y+kMR), the strip
//     keeping phi and the derived fields in rings of kMRing rows, so the y
//     halo of a strip is computed once per run of rows instead of per tile.
// HBM traffic per node and step is the algorithmic state (18 populations and
// phi u read and written); the x halo columns are re-read from L2 by the
// neighbouring strip.
//
// Supported: float32 and 16-bit storage, periodic or no-slip walls in y,
// periodic x with nx a multiple of the 16-byte chunk, every force form.
// Free-slip side walls, the macroscopic read-back and the taping step keep
// the tile kernels.
#pragma once

#include "step_kernel.cuh"

namespace pflbm {

constexpr int kMW = 64;                    // strip width (output columns)
constexpr int kMR = 4;                     // output rows per iteration
constexpr int kMRing = 8;                  // rows of the field rings (power of 2)
constexpr int kMThreads = 256;             // threads per CTA (8 warps)
constexpr int kMBlocks = 2;                // CTAs per SM

// wait until at most one committed group of this thread is still in flight
__device__ __forceinline__ void cp_async_wait_one() {
  asm volatile("cp.async.wait_group 1;" ::: "memory");
}

// Geometry of one row slot of the population ring for storage ST: h_0, then
// h_1..h_8 and f_0..f_8 (the "uniform" planes, in the storage type), then the
// two rows of (phi u)^{t-1}.  Column b of a population plane holds global
// column x0 - XP + b (XP: 16 bytes of halo), pulled for the node of the slot's
// row, i.e. storage row (row - c_iy) + 1.  Every plane row starts on a
// 16-byte boundary and spans a whole number of 16-byte chunks.
template <class ST>
struct MarchSlot {
  using T = typename ST::T;
  static constexpr int EB = sizeof(T);
  static constexpr int XP = 16 / EB;          // halo columns of a uniform plane
  static constexpr int PW = kMW + 2 * XP;     // columns of a uniform plane
  static constexpr int CE = 16 / EB;          // elements per 16-byte chunk
  static constexpr int XP0 = ST::kSplitH0 ? 4 : XP;  // h_0 (float32 when split)
  static constexpr int PW0 = kMW + 2 * XP0;
  static constexpr int H0B = ST::kSplitH0 ? PW0 * 4 : PW * EB;
  static constexpr int UB = PW * EB;          // bytes of a uniform plane row
  static constexpr int OFF_U = H0B;           // h_1..h_8, f_0..f_8
  static constexpr int OFF_PU = OFF_U + 17 * UB;
  static constexpr int CE0 = ST::kSplitH0 ? 4 : CE;  // elements of h_0 per chunk
  static constexpr int NCH0 = PW0 / CE0;             // 16-byte chunks of a row of h_0
  static constexpr int NCHU = PW / CE;               // ... of a uniform plane
  static constexpr int NCHP = kMW / 4;               // ... of a (phi u) row
  static constexpr int ROWCH = NCH0 + 17 * NCHU + 2 * NCHP;  // chunks of a node row
  static constexpr int BYTES = (OFF_PU + 2 * kMW * 4 + 127) / 128 * 128;
  // rows in use in an iteration (kMR + 3) and the two next iterations' new
  // rows in flight (2 kMR)
  static constexpr int SLOTS = 3 * kMR + 3;
  static_assert(PW % CE == 0 && H0B % 16 == 0 && UB % 16 == 0, "16-byte chunks");
  // uniform plane u: h_{u+1} for u < 8, f_{u-8} otherwise
  __device__ static int uoff(int u) { return OFF_U + u * UB; }
};

// Shared-memory field rings of the march (floats): phi on the strip + 3,
// the level-1 fields on the strip + 2, the level-2 fields on the strip + 1.
template <int FORM>
struct MarchFields {
  static constexpr int W3 = kMW + 6, W2 = kMW + 4, W1 = kMW + 2;
  static constexpr int NE = extra_fields<FORM>();
  static constexpr bool kLap = FORM == kPF1 || FORM == kPF2;
  static constexpr int NS2 = 3 + (kLap ? 1 : 0) + NE;  // grad phi, mu, [lap], [n]
  static constexpr int GX = 0, GY = 1, MU = 2, LAP = 3, E0 = kLap ? 4 : 3;
  static constexpr int FX = 0, FY = 1, UX = 2, UY = 3, PUX = 4, PUY = 5;
  static constexpr int OFF_PHI = 0;
  static constexpr int OFF_S2 = OFF_PHI + pad128(kMRing * W3 * 4);
  static constexpr int OFF_S1 = OFF_S2 + pad128(NS2 * kMRing * W2 * 4);
  static constexpr int BYTES = OFF_S1 + pad128(6 * kMRing * W1 * 4);
};

template <int FORM, class ST>
struct MarchSmem {
  using G = MarchSlot<ST>;
  using F = MarchFields<FORM>;
  static constexpr int OFF_RING = 0;
  static constexpr int OFF_FIELDS = OFF_RING + G::SLOTS * G::BYTES;
  static constexpr int BYTES = OFF_FIELDS + F::BYTES;
  static_assert(BYTES <= 113 * 1024, "two CTAs per SM");
};

// Central-scheme derivatives on three ring rows (rm = row - 1, r0, rp = row
// + 1), in the operation order of ics_dx / ics_dy.
__device__ __forceinline__ float ics3_dx(const float* rm, const float* r0, const float* rp, int c) {
  return (r0[c + 1] - r0[c - 1]) * (1.0f / 3.0f) +
         ((rp[c + 1] - rp[c - 1]) + (rm[c + 1] - rm[c - 1])) * (1.0f / 12.0f);
}
__device__ __forceinline__ float ics3_dy(const float* rm, const float* rp, int c) {
  return (rp[c] - rm[c]) * (1.0f / 3.0f) +
         ((rp[c + 1] - rm[c + 1]) + (rp[c - 1] - rm[c - 1])) * (1.0f / 12.0f);
}
template <class Fn>
__device__ __forceinline__ float ics3_dx_of(const Fn& a, int c) {  // a(drow, col)
  return (a(0, c + 1) - a(0, c - 1)) * (1.0f / 3.0f) +
         ((a(1, c + 1) - a(1, c - 1)) + (a(-1, c + 1) - a(-1, c - 1))) * (1.0f / 12.0f);
}
template <class Fn>
__device__ __forceinline__ float ics3_dy_of(const Fn& a, int c) {
  return (a(1, c) - a(-1, c)) * (1.0f / 3.0f) +
         ((a(1, c + 1) - a(-1, c + 1)) + (a(1, c - 1) - a(-1, c - 1))) * (1.0f / 12.0f);
}

__device__ __forceinline__ int ring_row(int r) { return r & (kMRing - 1); }

// The 16-byte chunks of a node row that one thread copies (at most two: a row
// has ROWCH chunks, the CTA kMThreads threads), fixed for a strip: chunk k
// reads storage row r of its plane at base[k] + r * pitch[k] and lands at
// byte dst[k] of the row's slot.  Population chunks read storage row
// (v - cy) + 1 for node row v; (phi u) chunks read row v (no ghost rows).
struct FillPlan {
  const unsigned char* base[2];
  int pitch[2], dst[2], cy[2], pu[2];
  int n;
};

template <class ST>
__device__ __forceinline__ FillPlan march_fill_plan(const StepArgs& a, int x0) {
  using G = MarchSlot<ST>;
  using T = typename ST::T;
  const Lattice& L = a.L;
  FillPlan pl;
  pl.n = 0;
  for (int c0 = threadIdx.x; c0 < G::ROWCH; c0 += kMThreads) {
    const int k = pl.n++;
    int c = c0;
    if (c < G::NCH0) {  // h_0
      const float* b = ST::kSplitH0 ? a.h0_in : reinterpret_cast<const float*>(a.h_in);
      pl.base[k] = reinterpret_cast<const unsigned char*>(b + wrap(x0 - G::XP0 + c * G::CE0, L.nx));
      pl.pitch[k] = L.nx * 4;
      pl.dst[k] = c * 16;
      pl.cy[k] = 0;
      pl.pu[k] = 0;
    } else if ((c -= G::NCH0) < 17 * G::NCHU) {  // h_1..h_8, f_0..f_8
      const int u = c / G::NCHU, j = c - u * G::NCHU;
      const int i = u < 8 ? u + 1 : u - 8;
      const T* b = u < 8 ? reinterpret_cast<const T*>(a.h_in) +
                               (size_t)(ST::kSplitH0 ? i - 1 : i) * L.plane
                         : reinterpret_cast<const T*>(a.f_in) + (size_t)i * L.plane;
      pl.base[k] = reinterpret_cast<const unsigned char*>(b + wrap(x0 - G::XP + j * G::CE, L.nx));
      pl.pitch[k] = L.nx * G::EB;
      pl.dst[k] = G::uoff(u) + j * 16;
      pl.cy[k] = qcy(i);
      pl.pu[k] = 0;
    } else {  // (phi u)^{t-1}
      c -= 17 * G::NCHU;
      const int comp = c / G::NCHP, j = c - comp * G::NCHP;
      pl.base[k] = reinterpret_cast<const unsigned char*>(
          a.phiu + (size_t)comp * L.nx * L.ny + wrap(x0 + 4 * j, L.nx));
      pl.pitch[k] = L.nx * 4;
      pl.dst[k] = G::OFF_PU + comp * kMW * 4 + j * 16;
      pl.cy[k] = 0;
      pl.pu[k] = 1;
    }
  }
  return pl;
}

// Issue this thread's copies of node row v into `slot`.  Population i of
// node row v is pulled from storage row (v - c_iy) + 1 (walls: the ghost rows
// hold the bounced populations; rows beyond a wall are not pulled and read as
// zero); periodic y wraps v - c_iy.
__device__ __forceinline__ void march_fill_row(const FillPlan& pl, const Lattice& L,
                                               unsigned char* slot, int v) {
  const bool inside = v >= 0 && v < L.ny;
  const bool valid = inside || !L.wall;
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    if (k >= pl.n) break;
    int r = v - pl.cy[k];
    if (!L.wall && (r < 0 || r >= L.ny)) r = wrap(r, L.ny);
    r += 1 - pl.pu[k];  // storage rows of the population planes start at the ghost row
    cp_async16(slot + pl.dst[k], pl.base[k] + (valid ? (size_t)r * pl.pitch[k] : 0), valid);
  }
}

template <int FORM, class ST>
__global__ void __launch_bounds__(kMThreads, kMBlocks)
    k_step_march(const __grid_constant__ StepArgs a) {
  using G = MarchSlot<ST>;
  using F = MarchFields<FORM>;
  using S = MarchSmem<FORM, ST>;
  using T = typename ST::T;
  constexpr int W3 = F::W3, W2 = F::W2, W1 = F::W1;
  constexpr bool kScaled = ST::kSplitH0;
  extern __shared__ __align__(128) unsigned char sm[];
  unsigned char* ring = sm + S::OFF_RING;
  float* sPhi = reinterpret_cast<float*>(sm + S::OFF_FIELDS + F::OFF_PHI);
  float* s2 = reinterpret_cast<float*>(sm + S::OFF_FIELDS + F::OFF_S2);
  float* s1 = reinterpret_cast<float*>(sm + S::OFF_FIELDS + F::OFF_S1);
  const Lattice& L = a.L;
  const Phys& P = a.p;
  const int tid = threadIdx.x;

  // this CTA's share: (strip, row) pairs [lo, hi) in strip-major order
  const int nstrips = (L.nx + kMW - 1) / kMW;
  const long long total = (long long)nstrips * L.ny;
  const long long lo = total * blockIdx.x / gridDim.x;
  const long long hi = total * (blockIdx.x + 1) / gridDim.x;

  const int nn = L.nx * L.ny;
  int seq_base = 0;  // sequence index (ring position) of the segment's first row
  for (long long w = lo; w < hi;) {
    const int strip = (int)(w / L.ny);
    const long long wend = hi < (long long)(strip + 1) * L.ny ? hi : (long long)(strip + 1) * L.ny;
    const int ya = (int)(w - (long long)strip * L.ny), yb = (int)(wend - (long long)strip * L.ny);
    const int niter = (yb - ya + kMR - 1) / kMR;
    const int vend = ya + niter * kMR + 3;
    const int x0 = strip * kMW;
    const auto seq_of = [&](int v) { return seq_base + (v - (ya - 3)); };
    const FillPlan plan = march_fill_plan<ST>(a, x0);
    const auto fill = [&](int v0, int v1) {  // rows of [v0, v1) that exist
      if (v1 > vend) v1 = vend;
      for (int v = v0; v < v1; ++v)
        march_fill_row(plan, L, ring + (seq_of(v) % G::SLOTS) * G::BYTES, v);
      cp_async_commit();
    };
    const auto slot_ptr = [&](int v) -> const unsigned char* {
      return ring + (seq_of(v) % G::SLOTS) * G::BYTES;
    };
    // population i of a slot at strip column b (node offset from x0), in the
    // storage scale
    const auto hpop = [&](const unsigned char* sl, int i, int b) -> float {
      if (i == 0) return reinterpret_cast<const float*>(sl)[b + G::XP0];
      return ST::raw(reinterpret_cast<const T*>(sl + G::uoff(i - 1))[b + G::XP - qcx(i)]);
    };
    const auto fpop = [&](const unsigned char* sl, int i, int b) -> float {
      return ST::raw(reinterpret_cast<const T*>(sl + G::uoff(8 + i))[b + G::XP - qcx(i)]);
    };
    const auto phi_row = [&](int v) { return sPhi + ring_row(v) * W3; };
    const auto s2_row = [&](int f, int v) { return s2 + (f * kMRing + ring_row(v)) * W2; };
    const auto s1_row = [&](int f, int v) { return s1 + (f * kMRing + ring_row(v)) * W1; };

    // A: phi on rows [r0, r1), strip columns -3 .. kMW + 2
    const auto stageA = [&](int r0, int r1) {
      const int n = (r1 - r0) * W3;
      for (int k = tid; k < n; k += kMThreads) {
        const int rr = k / W3, c = k - rr * W3;
        const int v = r0 + rr, b = c - 3;
        const unsigned char* sl = slot_ptr(v);
        float hh[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) hh[i] = hpop(sl, i, b);
        phi_row(v)[c] = phi_sum<ST>(hh, P);
      }
    };
    // walls: mirror ghosts of phi (row -k = row k - 1) for the rows of [r0, r1)
    // beyond a wall whose mirror row is still in the ring
    const auto mirror_phi = [&](int r0, int r1) {
      const int n = (r1 - r0) * W3;
      for (int k = tid; k < n; k += kMThreads) {
        const int rr = k / W3, c = k - rr * W3;
        const int v = r0 + rr;
        if (v >= 0 && v < L.ny) continue;
        const int m = map_row(v, L.ny, 1);
        if (m >= r1 - kMRing && m < r1) phi_row(v)[c] = phi_row(m)[c];
      }
    };
    // B: level-1 fields on rows [r0, r1), strip columns -2 .. kMW + 1
    const auto stageB = [&](int r0, int r1) {
      const int n = (r1 - r0) * W2;
      for (int k = tid; k < n; k += kMThreads) {
        const int rr = k / W2, c = k - rr * W2;
        const int v = r0 + rr, cc = c + 1;
        const float* pm = phi_row(v - 1);
        const float* p0 = phi_row(v);
        const float* pp = phi_row(v + 1);
        const float pc = p0[cc];
        const float gx = ics3_dx(pm, p0, pp, cc);
        const float gy = ics3_dy(pm, pp, cc);
        // Eq. ICS-sec: (2/cs^2) sum w_i (phi_i - phi_c)
        const float lap = ((p0[cc + 1] - pc) + (p0[cc - 1] - pc) + (pp[cc] - pc) + (pm[cc] - pc)) *
                              (2.0f / 3.0f) +
                          ((pp[cc + 1] - pc) + (pp[cc - 1] - pc) + (pm[cc + 1] - pc) +
                           (pm[cc - 1] - pc)) * (1.0f / 6.0f);
        s2_row(F::GX, v)[c] = gx;
        s2_row(F::GY, v)[c] = gy;
        if constexpr (F::kLap) s2_row(F::LAP, v)[c] = lap;
        s2_row(F::MU, v)[c] = P.beta4 * pc * ((pc - 1.0f) * (pc + 1.0f)) - P.kappa * lap;
        if constexpr (FORM == kCSF1 || FORM == kCSF2) {
          const float inv = rsqrtf(gx * gx + gy * gy + P.eps2);
          s2_row(F::E0, v)[c] = gx * inv;
          s2_row(F::E0 + 1, v)[c] = gy * inv;
        }
      }
    };
    // C: force, rho, u, phi u on rows [r0, r1), strip columns -1 .. kMW
    const auto stageC = [&](int r0, int r1) {
      const int n = (r1 - r0) * W1;
      for (int k = tid; k < n; k += kMThreads) {
        const int rr = k / W1, c = k - rr * W1;
        const int v = r0 + rr, b = c - 1, c2 = c + 1;
        const float phi = phi_row(v)[c + 2];
        const float gx = s2_row(F::GX, v)[c2], gy = s2_row(F::GY, v)[c2];
        float Fx, Fy;
        if constexpr (FORM == kSTF1 || FORM == kSTF2) {
          const float* gxr[3] = {s2_row(F::GX, v - 1), s2_row(F::GX, v), s2_row(F::GX, v + 1)};
          const float* gyr[3] = {s2_row(F::GY, v - 1), s2_row(F::GY, v), s2_row(F::GY, v + 1)};
          const auto txx = [&](int d, int cc) { return gxr[d + 1][cc] * gxr[d + 1][cc]; };
          const auto txy = [&](int d, int cc) { return gxr[d + 1][cc] * gyr[d + 1][cc]; };
          const auto tyy = [&](int d, int cc) { return gyr[d + 1][cc] * gyr[d + 1][cc]; };
          Fx = -P.kappa * (ics3_dx_of(txx, c2) + ics3_dy_of(txy, c2));
          Fy = -P.kappa * (ics3_dx_of(txy, c2) + ics3_dy_of(tyy, c2));
          if constexpr (FORM == kSTF2) {
            Fx += P.kappa * (ics3_dx_of(txx, c2) + ics3_dx_of(tyy, c2));
            Fy += P.kappa * (ics3_dy_of(txx, c2) + ics3_dy_of(tyy, c2));
          }
        } else if constexpr (FORM == kCPF1) {
          const float* m0 = s2_row(F::MU, v - 1);
          const float* m1 = s2_row(F::MU, v);
          const float* m2 = s2_row(F::MU, v + 1);
          Fx = -phi * ics3_dx(m0, m1, m2, c2);
          Fy = -phi * ics3_dy(m0, m2, c2);
        } else if constexpr (FORM == kCPF2) {
          const float mu = s2_row(F::MU, v)[c2];
          Fx = mu * gx;
          Fy = mu * gy;
        } else if constexpr (FORM == kPF1) {
          const float lap = s2_row(F::LAP, v)[c2];
          Fx = -P.kappa * gx * lap;
          Fy = -P.kappa * gy * lap;
        } else if constexpr (FORM == kPF2) {
          const float* l0 = s2_row(F::LAP, v - 1);
          const float* l1 = s2_row(F::LAP, v);
          const float* l2 = s2_row(F::LAP, v + 1);
          Fx = P.kappa * phi * ics3_dx(l0, l1, l2, c2);
          Fy = P.kappa * phi * ics3_dy(l0, l2, c2);
        } else {  // CSF-1, CSF-2
          const float divn = ics3_dx(s2_row(F::E0, v - 1), s2_row(F::E0, v), s2_row(F::E0, v + 1), c2) +
                             ics3_dy(s2_row(F::E0 + 1, v - 1), s2_row(F::E0 + 1, v + 1), c2);
          float coef;
          if constexpr (FORM == kCSF1) coef = -P.kappa * sqrtf(gx * gx + gy * gy) * divn;
          else coef = -P.half_sigma * divn;
          Fx = coef * gx;
          Fy = coef * gy;
        }
        const float rho = P.rho_mid + P.drho_half * phi;
        Fx += (rho - P.rho0) * P.gx;
        Fy += (rho - P.rho0) * P.gy;
        const unsigned char* sl = slot_ptr(v);
        float f[9];
#pragma unroll
        for (int i = 1; i < 9; ++i) f[i] = fpop(sl, i, b);
        float jx, jy;
        f_flux<ST>(f, P, jx, jy);
        // Eq. mac: u = [sum c f + cs^2 F / 2] / (cs^2 rho)
        const float irho = __fdividef(1.0f, rho);
        const float ux = (3.0f * jx + 0.5f * Fx) * irho;
        const float uy = (3.0f * jy + 0.5f * Fy) * irho;
        s1_row(F::FX, v)[c] = Fx;
        s1_row(F::FY, v)[c] = Fy;
        s1_row(F::UX, v)[c] = ux;
        s1_row(F::UY, v)[c] = uy;
        s1_row(F::PUX, v)[c] = phi * ux;
        s1_row(F::PUY, v)[c] = phi * uy;
      }
    };
    // walls: ghost of phi u beyond a wall, phi (2 u_w - u) of the mirrored node
    const auto ghost_phiu = [&](int r0, int r1) {
      for (int c = tid; c < W1; c += kMThreads) {
        if (r0 <= -1 && -1 < r1) {
          const float pm = phi_row(0)[c + 2];
          s1_row(F::PUX, -1)[c] = pm * (2.0f * P.uwb - s1_row(F::UX, 0)[c]);
          s1_row(F::PUY, -1)[c] = -pm * s1_row(F::UY, 0)[c];
        }
        if (r0 <= L.ny && L.ny < r1) {
          const float pm = phi_row(L.ny - 1)[c + 2];
          s1_row(F::PUX, L.ny)[c] = pm * (2.0f * P.uwt - s1_row(F::UX, L.ny - 1)[c]);
          s1_row(F::PUY, L.ny)[c] = -pm * s1_row(F::UY, L.ny - 1)[c];
        }
      }
    };
    // D: collide and store the nodes of rows [r0, r1)
    const auto stageD = [&](int r0, int r1) {
      const int n = (r1 - r0) * kMW;
      for (int k = tid; k < n; k += kMThreads) {
        const int rr = k / kMW, c = k - rr * kMW;
        const int gy = r0 + rr, gx = x0 + c;
        if (gx >= L.nx) continue;
        const unsigned char* sl = slot_ptr(gy);
        const float phi = phi_row(gy)[c + 3];
        const float Gx = s2_row(F::GX, gy)[c + 2], Gy = s2_row(F::GY, gy)[c + 2];
        const float mu = s2_row(F::MU, gy)[c + 2];
        const float Fx = s1_row(F::FX, gy)[c + 1], Fy = s1_row(F::FY, gy)[c + 1];
        const float ux = s1_row(F::UX, gy)[c + 1], uy = s1_row(F::UY, gy)[c + 1];
        const float rho = P.rho_mid + P.drho_half * phi;
        const float drx = P.drho_half * Gx, dry = P.drho_half * Gy;
        float f[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = fpop(sl, i, c);
        const float sumf = f_sum<ST>(f, P);
        // Eq. mac: P = sum f + cs^2/2 u . grad rho
        const float Pr = sumf + (ux * drx + uy * dry) * (1.0f / 6.0f);
        // div(phi u) by Eq. ICS-1st on the strip + 1 values
        const float div = ics3_dx(s1_row(F::PUX, gy - 1), s1_row(F::PUX, gy), s1_row(F::PUX, gy + 1), c + 1) +
                          ics3_dy(s1_row(F::PUY, gy - 1), s1_row(F::PUY, gy + 1), c + 1);
        const int n_idx = gy * L.nx + gx;
        const float pux = phi * ux, puy = phi * uy;
        float dtx = 0.0f, dty = 0.0f;
        if (!a.first) {
          const float* pu = reinterpret_cast<const float*>(sl + G::OFF_PU);
          dtx = pux - pu[c];
          dty = puy - pu[kMW + c];
        }
        if (!a.keep_phiu) {
          a.phiu[n_idx] = pux;
          a.phiu[nn + n_idx] = puy;
        }
        float h[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) h[i] = hpop(sl, i, c);

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
          for (int cl = 0; cl < 2; ++cl) {
            constexpr float wa = qw(1), wd = qw(5);
            const float wf = kScaled ? P.sf : (cl == 0 ? wa : wd);
            const float wh = kScaled ? P.sh : (cl == 0 ? wa : wd);
            K.t1[cl] = wf * oP;
            K.t2[cl] = wf * oR;
            K.t3[cl] = wf * cff;
            K.hc[cl] = wh * hb;
            K.hu[cl] = wh * hp;
            K.hd[cl] = wh * hd;
          }
        }
        float fo[9], ho[9];
        {
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

        if (L.wall && (gy == 0 || gy == L.ny - 1)) {
          // Ladd half-way bounce-back (Sec. 4) into the ghost rows, as in
          // step_tile (periodic x: the neighbour columns wrap)
          const int xr = gx + 1 < L.nx ? gx + 1 : 0;
          const int xl = gx - 1 >= 0 ? gx - 1 : L.nx - 1;
          const float bwf = kScaled ? P.sf : qw(7), bwh = kScaled ? P.sh : qw(7);
          if (gy == 0) {
            const float uw = P.uwb;
            store_fs<ST, 2>(a, gx, fo[4]);
            store_hs<ST, 2>(a, gx, ho[4]);
            store_fs<ST, 5>(a, xl, fo[7] - 2.0f * bwf * rho * (-uw));
            store_hs<ST, 5>(a, xl, ho[7] - 2.0f * bwh * phi * 3.0f * (-uw));
            store_fs<ST, 6>(a, xr, fo[8] - 2.0f * bwf * rho * uw);
            store_hs<ST, 6>(a, xr, ho[8] - 2.0f * bwh * phi * 3.0f * uw);
          }
          if (gy == L.ny - 1) {
            const float uw = P.uwt;
            const int g = (L.ny + 1) * L.nx;
            store_fs<ST, 4>(a, g + gx, fo[2]);
            store_hs<ST, 4>(a, g + gx, ho[2]);
            store_fs<ST, 7>(a, g + xr, fo[5] - 2.0f * bwf * rho * uw);
            store_hs<ST, 7>(a, g + xr, ho[5] - 2.0f * bwh * phi * 3.0f * uw);
            store_fs<ST, 8>(a, g + xl, fo[6] - 2.0f * bwf * rho * (-uw));
            store_hs<ST, 8>(a, g + xl, ho[6] - 2.0f * bwh * phi * 3.0f * (-uw));
          }
        }
      }
    };
    const auto outside = [&](int r0, int r1) { return L.wall && (r0 < 0 || r1 > L.ny); };

    // prologue: the rows of the prologue and of the first iteration, then
    // phi on [ya-3, ya+3), level-1 on [ya-2, ya+2), level-2 on [ya-1, ya+1)
    fill(ya - 3, ya + kMR + 3);
    fill(ya + kMR + 3, ya + 2 * kMR + 3);  // the second iteration's new rows
    cp_async_wait_one();
    __syncthreads();
    stageA(ya - 3, ya + 3);
    __syncthreads();
    if (outside(ya - 3, ya + 3)) {
      mirror_phi(ya - 3, ya + 3);
      __syncthreads();
    }
    stageB(ya - 2, ya + 2);
    __syncthreads();
    stageC(ya - 1, ya + 1);
    __syncthreads();
    if (outside(ya - 1, ya + 1)) {
      ghost_phiu(ya - 1, ya + 1);
      __syncthreads();
    }
    for (int it = 0; it < niter; ++it) {
      const int y = ya + it * kMR;
      // this iteration's rows landed (every group but the newest); then the
      // rows of the iteration after the next, into slots last used by rows
      // that every thread has finished with (the barrier ending the last
      // iteration)
      if (it > 0) {
        cp_async_wait_one();
        __syncthreads();
      }
      fill(y + 2 * kMR + 3, y + 3 * kMR + 3);
      stageA(y + 3, y + kMR + 3);
      __syncthreads();
      if (outside(y + 3, y + kMR + 3)) {
        mirror_phi(y + 3, y + kMR + 3);
        __syncthreads();
      }
      stageB(y + 2, y + kMR + 2);
      __syncthreads();
      stageC(y + 1, y + kMR + 1);
      __syncthreads();
      if (outside(y + 1, y + kMR + 1)) {
        ghost_phiu(y + 1, y + kMR + 1);
        __syncthreads();
      }
      stageD(y, y + kMR < yb ? y + kMR : yb);
      __syncthreads();
    }
    cp_async_wait_all();
    __syncthreads();
    seq_base += vend - (ya - 3);
    w = wend;
  }
}

template <int FORM, class ST>
cudaError_t launch_march(const StepArgs& a, cudaStream_t s) {
  using S = MarchSmem<FORM, ST>;
  static bool configured = false;
  if (!configured) {
    const cudaError_t e = cudaFuncSetAttribute(k_step_march<FORM, ST>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, S::BYTES);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const long long total = (long long)((a.L.nx + kMW - 1) / kMW) * a.L.ny;
  long long grid = (long long)num_sms() * kMBlocks;
  const long long most = total / (2 * kMR);  // at least two iterations per CTA
  if (grid > most) grid = most > 0 ? most : 1;
  k_step_march<FORM, ST><<<(int)grid, kMThreads, S::BYTES, s>>>(a);
  return cudaGetLastError();
}

}  // namespace pflbm

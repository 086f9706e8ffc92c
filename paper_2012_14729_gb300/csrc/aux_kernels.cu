// Initial state, population read-back and FP64 diagnostics of a domain.
#include "lattice.cuh"

namespace pflbm {

// Streaming multiprocessors of the current device (persistent grid size).
int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      n = v;
    else
      return 1;
  }
  return n;
}

// ---------------------------------------------------------------------------
// initial state (zero velocity, Sec. 5.1): f = f^eq(P = 0, u = 0) = 0 and
// h = h^eq(phi0, mu0, 0) with mu0 = 4 beta phi0 (phi0^2 - 1) - kappa lap phi0.
// The pre-collision value h_i(x) is written where the first pull reads it:
// population plane i at x - c_i (ghost rows for walls, wrapped otherwise;
// beyond a free-slip side wall, plane M, the mirror direction, in x's own
// column, where the specular pull reads).
// ---------------------------------------------------------------------------
template <class ST, int I, int M>
__device__ __forceinline__ void put_h(const StepArgs& a, int x, int y, float v) {
  const Lattice& L = a.L;
  int sx = x - qcx(I), sy = y - qcy(I);
  if (!L.wall) {
    if (sy < 0) sy += L.ny;
    if (sy >= L.ny) sy -= L.ny;
  }
  const int row = (sy + 1) * L.nx;
  if (sx < 0 || sx >= L.nx) {
    if (L.wall_x) {
      store_h<ST, M>(a, row + x, v);
      return;
    }
    sx = sx < 0 ? sx + L.nx : sx - L.nx;
  }
  store_h<ST, I>(a, row + sx, v);
}

template <class ST>
__global__ void k_init(const StepArgs a, const float* __restrict__ phi0) {
  const Lattice L = a.L;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= L.nx || y >= L.ny) return;
  auto at = [&](int dx, int dy) {
    return phi0[map_row(y + dy, L.ny, L.wall) * L.nx + map_col(x + dx, L.nx, L.wall_x)];
  };
  const float pc = at(0, 0);
  const float lap = ((at(1, 0) - pc) + (at(-1, 0) - pc) + (at(0, 1) - pc) + (at(0, -1) - pc)) *
                        (2.0f / 3.0f) +
                    ((at(1, 1) - pc) + (at(-1, 1) - pc) + (at(1, -1) - pc) + (at(-1, -1) - pc)) *
                        (1.0f / 6.0f);
  const float mu = a.p.beta4 * pc * ((pc - 1.0f) * (pc + 1.0f)) - a.p.kappa * lap;
  const float emu = a.p.eta * mu;
  put_h<ST, 0, 0>(a, x, y, pc + (qw(0) - 1.0f) * emu);
  put_h<ST, 1, 3>(a, x, y, qw(1) * emu);
  put_h<ST, 2, 2>(a, x, y, qw(2) * emu);
  put_h<ST, 3, 1>(a, x, y, qw(3) * emu);
  put_h<ST, 4, 4>(a, x, y, qw(4) * emu);
  put_h<ST, 5, 6>(a, x, y, qw(5) * emu);
  put_h<ST, 6, 5>(a, x, y, qw(6) * emu);
  put_h<ST, 7, 8>(a, x, y, qw(7) * emu);
  put_h<ST, 8, 7>(a, x, y, qw(8) * emu);
  const int n = L.nx * L.ny;
  a.phiu[y * L.nx + x] = 0.0f;
  a.phiu[n + y * L.nx + x] = 0.0f;
}

cudaError_t launch_init(int storage, const StepArgs& a, const float* phi0, cudaStream_t s) {
  dim3 grid((a.L.nx + 127) / 128, a.L.ny);
  switch (storage) {
    case kFP32: k_init<StoreF32><<<grid, 128, 0, s>>>(a, phi0); break;
    case kFP16: k_init<StoreF16><<<grid, 128, 0, s>>>(a, phi0); break;
    case kBF16: k_init<StoreBF16><<<grid, 128, 0, s>>>(a, phi0); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// decoded pre-collision populations [9][ny][nx]
// ---------------------------------------------------------------------------
template <class ST>
__global__ void k_read_pops(const StepArgs a, float* f_out, float* h_out) {
  const Lattice L = a.L;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= L.nx || y >= L.ny) return;
  const Pull q = L.wall_x ? pull_idx<true>(L, x, y) : pull_idx<false>(L, x, y);
  const int n = L.nx * L.ny, o = y * L.nx + x;
  float v[9];
  if (f_out) {
    pull_f<ST>(a, q, v);
#pragma unroll
    for (int i = 0; i < 9; ++i) f_out[i * n + o] = v[i];
  }
  if (h_out) {
    pull_h<ST>(a, q, v);
#pragma unroll
    for (int i = 0; i < 9; ++i) h_out[i * n + o] = v[i];
  }
}

cudaError_t launch_read_pops(int storage, const StepArgs& a, float* f_out, float* h_out,
                             cudaStream_t s) {
  dim3 grid((a.L.nx + 127) / 128, a.L.ny);
  switch (storage) {
    case kFP32: k_read_pops<StoreF32><<<grid, 128, 0, s>>>(a, f_out, h_out); break;
    case kFP16: k_read_pops<StoreF16><<<grid, 128, 0, s>>>(a, f_out, h_out); break;
    case kBF16: k_read_pops<StoreBF16><<<grid, 128, 0, s>>>(a, f_out, h_out); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 diagnostics: per-node terms accumulated in double, reduced by warp
// shuffles, then across warps in shared memory, one partial row per block;
// a single-block pass sums the partials in block order (deterministic).
// Slots: 0 sum phi, 1 max |u|^2, 2 area1 = sum w, 3 sum w x, 4 sum w y,
// 5 sum w x^2, 6 sum w y^2, 7 sum w x y, 8 sum p_in, 9 n_in, 10 sum p_out,
// 11 n_out, 12 non-finite count; w = (1 + phi)/2.
// ---------------------------------------------------------------------------
constexpr int kDiagThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Blocks take rows (grid-stride), threads take columns of a row; the y
// moments are formed once per row from the thread's row sums of w and w x,
// which keeps the FP64 work per node to the x moments (FP64 is slow here).
__global__ void __launch_bounds__(kDiagThreads) k_diag_partial(const Lattice L,
                                                               const float* __restrict__ fields,
                                                               const DiagGeom g,
                                                               double* __restrict__ partials) {
  const int n = L.nx * L.ny;
  double acc[13];
#pragma unroll
  for (int j = 0; j < 13; ++j) acc[j] = 0.0;
  for (int y = blockIdx.x; y < L.ny; y += gridDim.x) {
    const double yd = y;
    double rw = 0.0, rwx = 0.0;  // this thread's sums of w and w x over the row
    double dy = fabs(yd - g.yc);
    if (!L.wall) dy = fmin(dy, L.ny - dy);  // periodic distance across y
    const int row = y * L.nx;
    for (int x = threadIdx.x; x < L.nx; x += blockDim.x) {
      const int k = row + x;
      const float phif = fields[k], uxf = fields[2 * n + k], uyf = fields[3 * n + k];
      const float phf = fields[6 * n + k];
      if (!(isfinite(phif) && isfinite(uxf) && isfinite(uyf) && isfinite(phf) &&
            isfinite(fields[4 * n + k]))) {
        acc[12] += 1.0;
        continue;
      }
      const double phi = phif, ux = uxf, uy = uyf;
      const double w = 0.5 * (1.0 + phi);
      const double xd = x;
      acc[0] += phi;
      acc[1] = fmax(acc[1], ux * ux + uy * uy);
      rw += w;
      rwx += w * xd;
      acc[5] += w * xd * xd;
      if (g.has_geom) {
        double dx = fabs(xd - g.xc);
        if (!L.wall_x) dx = fmin(dx, L.nx - dx);  // periodic distance across x
        const double r = sqrt(dx * dx + dy * dy);
        const double ph = phf;
        if (r <= g.r_in) {
          acc[8] += ph;
          acc[9] += 1.0;
        }
        if (r >= g.r_out) {
          acc[10] += ph;
          acc[11] += 1.0;
        }
      }
    }
    acc[2] += rw;
    acc[3] += rwx;
    acc[4] += rw * yd;
    acc[6] += rw * yd * yd;
    acc[7] += rwx * yd;
  }
  __shared__ double red[kDiagThreads / 32][13];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < 13; ++j) {
    const double v = (j == 1) ? warp_max(acc[j]) : warp_sum(acc[j]);
    if (lane == 0) red[wid][j] = v;
  }
  __syncthreads();
  if (threadIdx.x < 13) {
    const int j = threadIdx.x;
    double v = red[0][j];
    for (int w = 1; w < kDiagThreads / 32; ++w) v = (j == 1) ? fmax(v, red[w][j]) : v + red[w][j];
    partials[blockIdx.x * kNRed + j] = v;
  }
}

// One warp per slot: lanes take block partials in a fixed stride and the
// warp combines them by shuffles (deterministic order).  Slots below nslots
// are summed, except max_slot (a maximum); the rest come out as 0.
__global__ void k_diag_final(const double* __restrict__ partials, int nblocks, int nslots,
                             int max_slot, double* __restrict__ out) {
  const int j = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (j >= kNRed) return;
  const bool is_max = j == max_slot;
  double v = 0.0;
  if (j < nslots)
    for (int b = lane; b < nblocks; b += 32) {
      const double p = partials[b * kNRed + j];
      v = is_max ? fmax(v, p) : v + p;
    }
  v = is_max ? warp_max(v) : warp_sum(v);
  if (lane == 0) out[j] = v;
}

// ---------------------------------------------------------------------------
// Rising-bubble quantities (Sec. 5.4).  Each thread takes nodes and, with
// each node, the lattice cell whose lower-left corner it is (cells wrap in a
// periodic direction; there is none beyond the last node towards a wall).
// Slots: 0 sum (1 - phi), 1 sum (1 - phi) x, 2 sum (1 - phi) y,
// 3 sum (1 - phi) u_x, 4 sum (1 - phi) u_y, 5 nodes with phi < 0,
// 6 phi = 0 contour length, 7 non-finite count.
// ---------------------------------------------------------------------------
constexpr int kBubbleSlots = 8;

// Contour length in one cell by marching squares.  Corners c0..c3 at
// (0,0), (1,0), (1,1), (0,1); inside means phi < 0; on an edge whose ends
// differ the contour passes the zero of the linear interpolant.  Four
// crossings (a saddle) are paired by the sign of the corner mean: inside,
// the segments cut off the two outside corners, else the two inside ones.
__device__ double cell_contour(double c0, double c1, double c2, double c3) {
  const bool i0 = c0 < 0.0, i1 = c1 < 0.0, i2 = c2 < 0.0, i3 = c3 < 0.0;
  const bool k0 = i0 != i1, k1 = i1 != i2, k2 = i2 != i3, k3 = i3 != i0;
  // crossing points, used only on cut edges: E0 on (0,0)-(1,0), E1 on
  // (1,0)-(1,1), E2 on (1,1)-(0,1), E3 on (0,1)-(0,0)
  const double e0x = c0 / (c0 - c1), e0y = 0.0;
  const double e1x = 1.0, e1y = c1 / (c1 - c2);
  const double e2x = 1.0 - c2 / (c2 - c3), e2y = 1.0;
  const double e3x = 0.0, e3y = 1.0 - c3 / (c3 - c0);
  if (k0 && k1 && k2 && k3) {
    const bool centre_in = ((c0 + c1) + c2) + c3 < 0.0;
    double len = 0.0;  // corner k lies between edges k-1 and k
    if (i0 != centre_in) len += hypot(e3x - e0x, e3y - e0y);
    if (i1 != centre_in) len += hypot(e0x - e1x, e0y - e1y);
    if (i2 != centre_in) len += hypot(e1x - e2x, e1y - e2y);
    if (i3 != centre_in) len += hypot(e2x - e3x, e2y - e3y);
    return len;
  }
  if (k0 && k1) return hypot(e0x - e1x, e0y - e1y);
  if (k0 && k2) return hypot(e0x - e2x, e0y - e2y);
  if (k0 && k3) return hypot(e0x - e3x, e0y - e3y);
  if (k1 && k2) return hypot(e1x - e2x, e1y - e2y);
  if (k1 && k3) return hypot(e1x - e3x, e1y - e3y);
  if (k2 && k3) return hypot(e2x - e3x, e2y - e3y);
  return 0.0;
}

__global__ void __launch_bounds__(kDiagThreads) k_bubble_partial(const Lattice L,
                                                                 const float* __restrict__ fields,
                                                                 double* __restrict__ partials) {
  const int n = L.nx * L.ny;
  double acc[kBubbleSlots];
#pragma unroll
  for (int j = 0; j < kBubbleSlots; ++j) acc[j] = 0.0;
  int inside = 0;  // nodes with phi < 0
  const float* __restrict__ phi = fields;
  // blocks take rows, threads take columns (y moment once per row)
  for (int y = blockIdx.x; y < L.ny; y += gridDim.x) {
    double rw = 0.0;
    const bool row_cells = y + 1 < L.ny || !L.wall;
    const int r0 = y * L.nx, r1 = (y + 1 < L.ny ? y + 1 : 0) * L.nx;
    for (int x = threadIdx.x; x < L.nx; x += blockDim.x) {
      const int k = r0 + x;
      const float pf = phi[k], uxf = fields[2 * n + k], uyf = fields[3 * n + k];
      if (!(isfinite(pf) && isfinite(uxf) && isfinite(uyf))) {
        acc[7] += 1.0;
        continue;
      }
      const double w = 1.0 - (double)pf;
      rw += w;
      acc[1] += w * x;
      acc[3] += w * (double)uxf;
      acc[4] += w * (double)uyf;
      inside += pf < 0.0f ? 1 : 0;
      if (row_cells && (x + 1 < L.nx || !L.wall_x)) {
        const int x1 = x + 1 < L.nx ? x + 1 : 0;
        const float c1 = phi[r0 + x1], c2 = phi[r1 + x1], c3 = phi[r1 + x];
        // a non-finite corner is counted at its own node; its cells add nothing
        const float lo = fminf(fminf(pf, c1), fminf(c2, c3));
        const float hi = fmaxf(fmaxf(pf, c1), fmaxf(c2, c3));
        if (lo < 0.0f && hi >= 0.0f && isfinite(c1) && isfinite(c2) && isfinite(c3))
          acc[6] += cell_contour(pf, c1, c2, c3);
      }
    }
    acc[0] += rw;
    acc[2] += rw * y;
  }
  acc[5] = inside;
  __shared__ double red[kDiagThreads / 32][kBubbleSlots];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < kBubbleSlots; ++j) {
    const double v = warp_sum(acc[j]);
    if (lane == 0) red[wid][j] = v;
  }
  __syncthreads();
  if (threadIdx.x < kBubbleSlots) {
    const int j = threadIdx.x;
    double v = red[0][j];
    for (int w = 1; w < kDiagThreads / 32; ++w) v += red[w][j];
    partials[blockIdx.x * kNRed + j] = v;
  }
}


// one block per row, up to max_blocks (then rows grid-stride)
int row_blocks(int ny, int max_blocks) { return ny < max_blocks ? (ny > 0 ? ny : 1) : max_blocks; }

cudaError_t launch_diag(const Lattice& L, const float* fields, DiagGeom g, double* partials,
                        int max_blocks, double* red, cudaStream_t s) {
  const int nb = row_blocks(L.ny, max_blocks);
  k_diag_partial<<<nb, kDiagThreads, 0, s>>>(L, fields, g, partials);
  k_diag_final<<<1, 32 * kNRed, 0, s>>>(partials, nb, 13, 1, red);
  return cudaGetLastError();
}

cudaError_t launch_bubble_diag(const Lattice& L, const float* fields, double* partials,
                               int max_blocks, double* red, cudaStream_t s) {
  const int nb = row_blocks(L.ny, max_blocks);
  k_bubble_partial<<<nb, kDiagThreads, 0, s>>>(L, fields, partials);
  k_diag_final<<<1, 32 * kNRed, 0, s>>>(partials, nb, kBubbleSlots, -1, red);
  return cudaGetLastError();
}

}  // namespace pflbm

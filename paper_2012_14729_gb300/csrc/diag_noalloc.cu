// FP64 field diagnostics that allocate nothing: the reduction scratch is a
// file-scope device array of fixed size instead of caller or workspace
// memory.  The per-node terms and both reduction stages are those of the
// workspace diagnostics (one partial row per 256-node block, then one warp
// per slot over the rows in a fixed lane stride); here the two stages run in
// one launch, the last block to finish taking the final stage.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "pflbm.h"
#include "internal.h"

namespace pflbm {
namespace {

constexpr int kThreads = 256;                       // nodes per block (one per thread)
constexpr int kRows = PFLBM_NOALLOC_MAX_NODES / kThreads;  // partial rows held
static_assert(kRows * kThreads == PFLBM_NOALLOC_MAX_NODES, "whole blocks");
constexpr int kRedOff = kRows * kNRed;               // final slots (doubles)
constexpr int kTicketOff = kRedOff + kNRed;          // block-completion counter
constexpr int kScratchDoubles = kTicketOff + 16;     // 128 bytes for the counter

// partials [kRows][kNRed] | red [kNRed] | ticket (unsigned int) : 4 MiB + 256 B
static __device__ __align__(256) double g_scratch[kScratchDoubles];

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

// Slots: 0 sum phi, 1 max |u|^2, 2 sum w, 3 sum w x, 4 sum w y, 5 sum w x^2,
// 6 sum w y^2, 7 sum w x y, 8 sum p_h inside, 9 n inside, 10 sum p_h outside,
// 11 n outside, 12 non-finite count; w = (1 + phi)/2 (Secs. 5.1, 5.2, 5.5).
// wrap_x / wrap_y: the lattice is periodic in that direction, so the
// distance to the pressure-jump centre is the periodic one there.
__global__ void __launch_bounds__(kThreads)
    k_diag_noalloc(const int nx, const int ny, const int wrap_x, const int wrap_y,
                   const float* __restrict__ fields, const DiagGeom g,
                   double* __restrict__ scratch) {
  const int n = nx * ny;
  double acc[13];
#pragma unroll
  for (int j = 0; j < 13; ++j) acc[j] = 0.0;
  const int k = blockIdx.x * kThreads + threadIdx.x;
  if (k < n) {
    const int y = k / nx, x = k - y * nx;
    const double phi = fields[k];
    const double ux = fields[2 * n + k], uy = fields[3 * n + k];
    const double ph = fields[6 * n + k];
    const bool finite = isfinite(phi) && isfinite(ux) && isfinite(uy) && isfinite(ph) &&
                        isfinite((double)fields[4 * n + k]);
    if (!finite) {
      acc[12] += 1.0;
    } else {
      const double w = 0.5 * (1.0 + phi);
      acc[0] += phi;
      acc[1] = fmax(acc[1], ux * ux + uy * uy);
      acc[2] += w;
      acc[3] += w * x;
      acc[4] += w * y;
      acc[5] += w * x * x;
      acc[6] += w * y * y;
      acc[7] += w * x * y;
      if (g.has_geom) {
        double dx = fabs(x - g.xc), dy = fabs(y - g.yc);
        if (wrap_x) dx = fmin(dx, nx - dx);
        if (wrap_y) dy = fmin(dy, ny - dy);
        const double r = sqrt(dx * dx + dy * dy);
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
  }
  __shared__ double red[kThreads / 32][13];
  __shared__ int is_last;
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
    for (int w = 1; w < kThreads / 32; ++w) v = (j == 1) ? fmax(v, red[w][j]) : v + red[w][j];
    scratch[blockIdx.x * kNRed + j] = v;
    __threadfence();  // the row is visible device-wide before the ticket is taken
  }
  __syncthreads();
  unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch + kTicketOff);
  if (threadIdx.x == 0) is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!is_last) return;
  // final stage: every row is written; read them from L2 (not this SM's L1)
  __threadfence();
  const int nrows = gridDim.x;
  for (int j = wid; j < kNRed; j += kThreads / 32) {
    double v = 0.0;
    if (j < 13)
      for (int b = lane; b < nrows; b += 32) {
        const double p = __ldcg(scratch + b * kNRed + j);
        v = (j == 1) ? fmax(v, p) : v + p;
      }
    v = (j == 1) ? warp_max(v) : warp_sum(v);
    if (lane == 0) scratch[kRedOff + j] = v;
  }
  if (threadIdx.x == 0) *ticket = 0u;  // ready for the next call
}

// Device address of the scratch array on the current device.  It is looked
// up on every call: the first lookup on a device loads this file's module
// there (which reserves the array), later ones find the loaded module.  A
// cached address would go stale when the application resets the device,
// since the module is then loaded again, possibly elsewhere.
cudaError_t scratch_address(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

// Same conversion of the reduced slots as pflbm_diagnostics.
void to_diag(const double* h, int has_geom, pflbm_diag* out) {
  memset(out, 0, sizeof(*out));
  out->mass = h[0];
  out->umax = sqrt(h[1]);
  out->area1 = h[2];
  out->R_num = sqrt(h[2] / M_PI);
  if (has_geom && h[9] > 0 && h[11] > 0) {
    out->p_in = h[8] / h[9];
    out->p_out = h[10] / h[11];
    out->dp = out->p_in - out->p_out;
    out->sigma_num = out->R_num * out->dp;
  }
  if (h[2] > 0) {
    const double cx = h[3] / h[2], cy = h[4] / h[2];
    out->xc1 = cx;
    out->yc1 = cy;
    const double sxx = h[5] / h[2] - cx * cx, syy = h[6] / h[2] - cy * cy;
    const double sxy = h[7] / h[2] - cx * cy;
    const double tr = sxx + syy, det = sxx * syy - sxy * sxy;
    const double disc = sqrt(fmax(tr * tr / 4 - det, 0.0));
    const double l1 = tr / 2 + disc, l2 = fmax(tr / 2 - disc, 0.0);
    const double Lx = 4 * sqrt(l1), Bx = 4 * sqrt(l2);
    out->taylor_D = (Lx + Bx) > 0 ? (Lx - Bx) / (Lx + Bx) : 0.0;
  }
  out->nonfinite = h[12];
}

pflbm_status cuda_fail(const char* what, cudaError_t e) {
  char msg[384];
  snprintf(msg, sizeof(msg), "pflbm_field_diagnostics_noalloc: %s: %s (%s)", what,
           cudaGetErrorName(e), cudaGetErrorString(e));
  set_last_error(msg);
  return PFLBM_ECUDA;
}

}  // namespace
}  // namespace pflbm

using namespace pflbm;

extern "C" pflbm_status pflbm_field_diagnostics_noalloc(int nx, int ny, pflbm_bc bc_x,
                                                        pflbm_bc bc_y, const float* fields,
                                                        const pflbm_diag_geom* geom,
                                                        pflbm_diag* out, void* stream) {
  char msg[384];
  if (nx <= 0 || ny <= 0 || !fields || !out) {
    set_last_error("pflbm_field_diagnostics_noalloc: nx, ny must be positive and fields, out "
                   "non-null");
    return PFLBM_EINVAL;
  }
  if ((bc_x != PFLBM_PERIODIC && bc_x != PFLBM_FREESLIP) ||
      (bc_y != PFLBM_PERIODIC && bc_y != PFLBM_WALL)) {
    set_last_error("pflbm_field_diagnostics_noalloc: bc_x must be PFLBM_PERIODIC or "
                   "PFLBM_FREESLIP, bc_y PFLBM_PERIODIC or PFLBM_WALL");
    return PFLBM_EINVAL;
  }
  const long long n = (long long)nx * ny;
  if (n > PFLBM_NOALLOC_MAX_NODES) {
    snprintf(msg, sizeof(msg),
             "pflbm_field_diagnostics_noalloc: a %d x %d lattice has %lld nodes; the static "
             "scratch holds partial sums for at most %d nodes",
             nx, ny, n, PFLBM_NOALLOC_MAX_NODES);
    set_last_error(msg);
    return PFLBM_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail("current device", e);
  cudaPointerAttributes pa;
  e = cudaPointerGetAttributes(&pa, fields);
  if (e != cudaSuccess) return cuda_fail("fields pointer", e);
  if ((pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) ||
      (pa.type == cudaMemoryTypeDevice && pa.device != dev)) {
    set_last_error("pflbm_field_diagnostics_noalloc: fields must be device memory of the "
                   "current device");
    return PFLBM_EINVAL;
  }
  double* scratch = nullptr;
  e = scratch_address(&scratch);
  if (e != cudaSuccess) return cuda_fail("scratch address", e);

  const cudaStream_t s = static_cast<cudaStream_t>(stream);
  DiagGeom g = {0, 0, 0, 0, 0};
  if (geom) g = DiagGeom{geom->xc, geom->yc, geom->r_in, geom->r_out, 1};
  const int nb = (int)((n + kThreads - 1) / kThreads);
  // the block-completion counter must start at zero
  e = cudaMemsetAsync(scratch + kTicketOff, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return cuda_fail("clear counter", e);
  k_diag_noalloc<<<nb, kThreads, 0, s>>>(nx, ny, bc_x == PFLBM_PERIODIC, bc_y == PFLBM_PERIODIC,
                                         fields, g, scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail("launch", e);
  double h[kNRed];
  e = cudaMemcpyAsync(h, scratch + kRedOff, sizeof(h), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail("read result", e);
  to_diag(h, g.has_geom, out);
  return h[12] > 0 ? PFLBM_EUNSTABLE : PFLBM_OK;
}

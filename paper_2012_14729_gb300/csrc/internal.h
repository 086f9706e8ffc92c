// Internal declarations of the CUDA library behind include/pflbm.h.
// Host-side argument blocks of the kernels and the per-storage launchers.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace pflbm {

constexpr int kNQ = 9;
constexpr int kNFields = 9;   // phi, rho, ux, uy, P, mu, p_h, Fx, Fy
constexpr int kNRed = 16;     // FP64 reduction slots of the diagnostics

enum Storage { kFP32 = 0, kFP16 = 1, kBF16 = 2 };

// Physical constants of one domain, precomputed in double on the host and
// rounded once to float (Sec. 2.1 and Sec. 3 of the paper).
struct Phys {
  float beta4;       // 4 beta, beta = 3 sigma / (4 W)
  float kappa;       // 3 W sigma / 8
  float half_sigma;  // sigma / 2 (CSF-2)
  float eps2;        // eps^2 of the CSF normal
  float rho_mid;     // (rho1 + rho2) / 2:  rho = rho_mid + drho_half phi
  float drho_half;   // (rho1 - rho2) / 2:  grad rho = drho_half grad phi
  float mu_mid;      // (rho1 nu1 + rho2 nu2) / 2: dynamic viscosity mid value
  float mu_dhalf;    // (rho1 nu1 - rho2 nu2) / 2
  float gx, gy, rho0;
  float uwb, uwt;    // x-velocity of the bottom / top wall
  float inv_tau_h;   // 1 / tau_h
  float hforce;      // 1 - 1 / (2 tau_h)
  float eta;         // M / (cs^2 (tau_h - 1/2))
  float acoef;       // 3 tau2 / (tau_h tau1)
  float sf, inv_sf;  // 16-bit storage scales of f
  float sh, inv_sh;  // and of h_1..h_8
};

struct Lattice {
  int nx, ny;
  int wall;          // 1: half-way bounce-back walls at y = -1/2, ny - 1/2
  int plane;         // elements per population plane: (ny + 2) * nx
  int wall_x;        // 1: free-slip (mirror-symmetry) walls at x = -1/2, nx - 1/2
};

// Arguments of one fused step (or macroscopic read) over one domain.  The
// tensor maps describe the input population arrays as 2-D tensors of
// nplanes * (ny + 2) rows of nx elements, for TMA box loads.
struct StepArgs {
  CUtensorMap tm_f;   // f_in (9 planes)
  CUtensorMap tm_h;   // h_in (9 planes, or 8 planes h_1..h_8 for 16-bit storage)
  CUtensorMap tm_h0;  // h0_in (16-bit storage only)
  int use_tma;        // tensor maps valid and row pitch 16-byte aligned
  int* err;           // device error word: bit 0 = a bounded wait expired
  Lattice L;
  Phys p;
  const void* f_in;   // post-collision populations of the previous step
  void* f_out;        // written by this step
  const void* h_in;   // FP32: 9 planes; 16-bit: planes of h_1..h_8
  void* h_out;
  const float* h0_in; // 16-bit storage only: h_0 in float32
  float* h0_out;
  float* phiu;        // [2][ny][nx]: in (phi u)^{t-1}, out (phi u)^t
  float* fields;      // macro mode: [kNFields][ny][nx]
  int first;          // first step of a run: d_t(phi u) = 0
  int macro;          // 1: write fields instead of colliding
  int keep_phiu;      // 1: do not write (phi u)^t back (autotuning trial steps)
  float* tape;        // taping step only: [kTapePlanes][ny][nx] of this step
};

// Planes the taping step records per node for the adjoint: the pulled f, then
// phi, grad phi, lap phi, mu, the force-form values A0/A1 (STF: F_sf; CPF-1:
// grad mu; PF-2: grad lap phi; CSF: div n), the total force, u, P, div(phi u)
// and d_t(phi u).
enum TapePlane {
  TP_F0 = 0, TP_PHI = 9, TP_GX, TP_GY, TP_L, TP_MU, TP_A0, TP_A1, TP_FX, TP_FY, TP_UX, TP_UY,
  TP_PR, TP_DIV, TP_DTX, TP_DTY, kTapePlanes
};

// Tile of the fused step kernel.
constexpr int kTX = 32;
constexpr int kTY = 16;
// Rows of the short tiles a gather-mode batch may run instead (one collision
// node per thread of a 256-thread CTA).
constexpr int kShortRows = 8;
// How a tile gets the populations it pulls (the autotuner picks per domain):
//   kBoxes   TMA box loads into shared memory (cp.async for seam tiles); a
//            persistent grid of two 512-thread CTAs per SM, each walking tiles
//   kGather  direct L1-cached gathers from global memory; one 256-thread CTA
//            per tile, four CTAs per SM
//   kMarch   column strips swept along y by persistent CTAs, the pulled
//            population rows staged ahead into a shared-memory ring by
//            cp.async (march_kernel.cuh); single domains only, periodic x
//            with nx a multiple of the 16-byte chunk, no side walls
//   kGather8 the gathers on tiles of kShortRows rows, one collision node per
//            thread of a 256-thread CTA, whose own node's populations stay in
//            registers from the pull to the collision; four CTAs per SM
enum StageMode { kBoxes = 0, kGather = 1, kMarch = 2, kGather8 = 3, kNumModes = 4 };
constexpr int kNumBatchModes = 2;  // the batch stages by boxes or gathers
constexpr int kThreadsBoxes = 512;
constexpr int kThreadsGather = 256;
constexpr int kBlocksBoxes = 2;   // CTAs per SM the box kernel is built for
constexpr int kBlocksGather = 4;
// Spin limit of the kernel's mbarrier waits (each try_wait suspends for a
// hardware-bounded time); past it the kernel flags err and returns.
constexpr long long kWaitLimit = 1ll << 20;

// Box geometry of the TMA loads for a storage element size: columns
// [x0 - xpad, x0 + kTX + xpad) so that the start column is 16-byte aligned.
__host__ __device__ constexpr int box_xpad(int elem_bytes) { return 16 / elem_bytes; }
__host__ __device__ constexpr int box_w(int elem_bytes) { return kTX + 2 * box_xpad(elem_bytes); }
constexpr int kBoxRowsH = kTY + 6;  // phi is needed on the tile + 3 ring
constexpr int kBoxRowsF = kTY + 2;  // f on the tile + 1 ring

// Adjoint of one step (adjoint.cu), float32 planes of n = nx ny nodes.
// Adjoint state between reverse steps: first one float4 per node of scalars
// (SB, JX, JY, PHI) that are added to every population when it is read (f_i:
// AP_F0 + i + SB + c_i . (JX, JY); h_i: AP_H0 + i + PHI), then the
// per-population planes and the adjoint of (phi u)^{t-1}; plane p starts at
// float offset (kAdjScalar + p) n.
enum AdjPlane { AP_F0 = 0, AP_H0 = 9, AP_QX = 18, AP_QY, kAdjPlanes };
constexpr int kAdjScalar = 4;  // floats of the per-node scalar block
// Work planes of one reverse step.
enum WorkPlane {
  B_PHI, B_RHO, B_UX, B_UY, B_P, B_FX, B_FY, B_GX, B_GY, B_MU, B_DIV, B_DTX, B_DTY, B_L,
  kWorkPlanes
};
struct AdjGeo {
  int nx, ny, wall;
};
struct AdjArgs {
  AdjGeo g;
  Phys p;
  int form, first;
  const float* tape;  // [kTapePlanes][n] recorded by the taping step at t
  const float* ain;   // adjoint state at t + 1: float4 [n], then [kAdjPlanes][n]
  float* aout;        // adjoint state at t, same layout
  float* W;           // [kWorkPlanes][n]
  double* acc;        // [4]: d/d(4 beta), d/d kappa, d/d eta, direct d/d sigma
};
// Taping step (the plain step plus the record of its intermediates in a.tape);
// setup_tape_step sets its kernel attributes and must precede a capture.
cudaError_t setup_tape_step(int form);
cudaError_t launch_tape_step(int form, const StepArgs& a, cudaStream_t s);
// Reverse of one step: 2 kernels.
cudaError_t launch_adjoint_step(const AdjArgs& A, cudaStream_t s);
// Adjoint of the initial state h = h^eq(phi0, mu0, 0): dphi0 from A.ain.
cudaError_t launch_adjoint_init(const AdjArgs& A, const float* phi0, float* dphi0,
                                cudaStream_t s);

// Batched step over a work-list (batch.cu): table holds 2 StepArgs per
// instance (entry 2 i + p reads buffer cur_i ^ p), items (instance, x0, y0,
// form) for tiles of `rows` rows (kTY, or kShortRows in the gather mode);
// `bp` is the step parity; `grid` persistent CTAs, which claim the items
// through the device counter `tickets` (zeroed on the stream before the
// kernel).
int batch_blocks_per_sm(int mode);
int num_sms();  // streaming multiprocessors of the current device
cudaError_t launch_batch(int mode, int rows, const StepArgs* table, const int4* items,
                         int nitems, int bp, int grid, unsigned* tickets, cudaStream_t s);

cudaError_t launch_step_fp32(int form, int mode, const StepArgs& a, cudaStream_t s);
cudaError_t launch_step_fp16(int form, int mode, const StepArgs& a, cudaStream_t s);
cudaError_t launch_step_bf16(int form, int mode, const StepArgs& a, cudaStream_t s);

// Initial state from phi0 (device, [ny][nx]).
cudaError_t launch_init(int storage, const StepArgs& a, const float* phi0, cudaStream_t s);
// Decoded pre-collision populations (either output may be null).
cudaError_t launch_read_pops(int storage, const StepArgs& a, float* f_out, float* h_out,
                             cudaStream_t s);

struct DiagGeom {
  double xc, yc, r_in, r_out;
  int has_geom;
};
// FP64 reductions of the staged fields into red[kNRed] (partials in scratch).
cudaError_t launch_diag(const Lattice& L, const float* fields, DiagGeom g, double* partials,
                        int max_blocks, double* red, cudaStream_t s);
// Rising-bubble sums of the staged fields (fluid-2 moments, phi < 0 count,
// marching-squares contour length) into red[0..7].
cudaError_t launch_bubble_diag(const Lattice& L, const float* fields, double* partials,
                               int max_blocks, double* red, cudaStream_t s);

// Message returned by pflbm_last_error() on this thread.
void set_last_error(const char* msg);

}  // namespace pflbm

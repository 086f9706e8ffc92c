// Host side of the C ABI declared in include/pflbm.h: workspace layout,
// parameter checks, launches on the caller's stream, CUDA graph replay,
// read-back, diagnostics and checkpoints.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "pflbm.h"
#include <cudaTypedefs.h>

#include "internal.h"

using namespace pflbm;

namespace {

thread_local char g_err[512] = "";

void set_err(const char* what, cudaError_t e) {
  snprintf(g_err, sizeof(g_err), "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}
void set_msg(const char* msg) { snprintf(g_err, sizeof(g_err), "%s", msg); }

constexpr size_t kAlign = 256;
constexpr int kMaxDiagBlocks = 1024;
// state blob magics: without / with the mean of phi0 in the header
constexpr long long kStateMagic = 0x70666c626d;
constexpr long long kStateMagicMean = 0x70666c626e;
constexpr int kGraphSteps = 64;  // steps captured per graph (even)

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

size_t elem_bytes(int storage) { return storage == kFP32 ? 4 : 2; }

struct Layout {
  size_t f[2], h[2], h0[2], phiu, fields, partials, red, err, total;
};

bool layout_of(int nx, int ny, int storage, Layout* L) {
  if (nx < 4 || ny < 4 || storage < 0 || storage > 2) return false;
  const size_t plane = (size_t)(ny + 2) * nx;
  if (plane * 9 >= (size_t)1 << 31) return false;
  const size_t n = (size_t)nx * ny;
  const size_t eb = elem_bytes(storage);
  const bool split = storage != kFP32;
  size_t off = 0;
  for (int b = 0; b < 2; ++b) {
    L->f[b] = off;
    off = align_up(off + 9 * plane * eb);
    L->h[b] = off;
    off = align_up(off + (split ? 8 : 9) * plane * eb);
    L->h0[b] = off;
    off = align_up(off + (split ? plane * 4 : 0));
  }
  L->phiu = off;
  off = align_up(off + 2 * n * 4);
  L->fields = off;
  off = align_up(off + (size_t)kNFields * n * 4);
  L->partials = off;
  off = align_up(off + (size_t)kMaxDiagBlocks * kNRed * 8);
  L->red = off;
  off = align_up(off + kNRed * 8);
  L->err = off;
  off = align_up(off + 4);
  L->total = off;
  return true;
}

}  // namespace

void pflbm::set_last_error(const char* msg) { set_msg(msg); }

struct pflbm_domain {
  int nx, ny, wall, storage;
  int wall_x;  // free-slip side walls
  cudaStream_t stream;
  char* ws;
  Layout lay;
  int cur;  // buffer holding the current post-collision state
  long long t;
  int has_params, has_state;
  pflbm_params par;
  Phys phys;
  // TMA descriptors of the input population arrays of each buffer
  CUtensorMap tm_f[2], tm_h[2], tm_h0[2];
  int use_tma;  // maps built and usable
  int tma_off;  // caller asked for plain loads
  int mode;     // StageMode of the step kernel
  int graphs;
  cudaGraphExec_t gexec;
  int g_parity;  // buffer parity the captured graph starts from
  // mean of phi0 over the lattice (the run's initial condition), from which
  // the default background density rho0 = rho(mean phi0) follows
  int has_mean_phi0;
  double mean_phi0;
};

namespace {

// rho is linear in phi, so the mean initial density is rho(mean phi0)
float default_rho0(const pflbm_domain* d) {
  const double m = d->mean_phi0;
  return (float)(0.5 * d->par.rho1 * (1 + m) + 0.5 * d->par.rho2 * (1 - m));
}

bool is_pow2(double v) {
  if (!(v > 0) || !isfinite(v)) return false;
  int e;
  double m = frexp(v, &e);
  return m == 0.5;
}

StepArgs make_args(const pflbm_domain* d, int from) {
  StepArgs a;
  memset(&a, 0, sizeof(a));
  a.L.nx = d->nx;
  a.L.ny = d->ny;
  a.L.wall = d->wall;
  a.L.wall_x = d->wall_x;
  a.L.plane = (d->ny + 2) * d->nx;
  a.p = d->phys;
  const int to = 1 - from;
  a.f_in = d->ws + d->lay.f[from];
  a.f_out = d->ws + d->lay.f[to];
  a.h_in = d->ws + d->lay.h[from];
  a.h_out = d->ws + d->lay.h[to];
  if (d->storage != kFP32) {
    a.h0_in = reinterpret_cast<const float*>(d->ws + d->lay.h0[from]);
    a.h0_out = reinterpret_cast<float*>(d->ws + d->lay.h0[to]);
  }
  a.phiu = reinterpret_cast<float*>(d->ws + d->lay.phiu);
  a.fields = reinterpret_cast<float*>(d->ws + d->lay.fields);
  a.err = reinterpret_cast<int*>(d->ws + d->lay.err);
  a.use_tma = d->use_tma && !d->tma_off;
  if (a.use_tma) {
    a.tm_f = d->tm_f[from];
    a.tm_h = d->tm_h[from];
    a.tm_h0 = d->tm_h0[from];
  }
  return a;
}

// cuTensorMapEncodeTiled from the driver, resolved once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// A [planes * rows][nx] array as a 2-D tensor with boxes of box_rows rows of
// box_cols columns.  Every box of a domain has the column count of its
// population storage (box_w of the 16-bit element for FP16/BF16, also for the
// float32 h_0 plane), matching the kernel's shared-memory geometry.
bool encode_map(CUtensorMap* m, void* base, CUtensorMapDataType dt, int elem, int nx,
                long long rows, int box_cols, int box_rows) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)nx, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)nx * elem};
  cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(m, dt, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor maps of both buffers; TMA is used only when the row pitch is a
// multiple of 16 bytes and the grid is wide enough for interior tiles.
void build_maps(pflbm_domain* d) {
  d->use_tma = 0;
  const int eb = (int)elem_bytes(d->storage);
  if ((d->nx * eb) % 16 != 0) return;
  const CUtensorMapDataType dt = d->storage == kFP32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : d->storage == kFP16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                       : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  const long long rows = d->ny + 2;
  const bool split = d->storage != kFP32;
  bool ok = true;
  const int bw = box_w(eb);
  for (int b = 0; b < 2 && ok; ++b) {
    ok = encode_map(&d->tm_f[b], d->ws + d->lay.f[b], dt, eb, d->nx, 9 * rows, bw, kBoxRowsF) &&
         encode_map(&d->tm_h[b], d->ws + d->lay.h[b], dt, eb, d->nx, (split ? 8 : 9) * rows, bw,
                    kBoxRowsH);
    if (ok && split)
      ok = encode_map(&d->tm_h0[b], d->ws + d->lay.h0[b], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4,
                      d->nx, rows, bw, kBoxRowsH);
    if (ok && !split) d->tm_h0[b] = d->tm_h[b];
  }
  d->use_tma = ok ? 1 : 0;
}

// The marching stage mode handles this domain: periodic x in whole 16-byte
// chunks of the storage type, no side walls, at least 8 rows.
bool march_ok(const pflbm_domain* d) {
  return !d->wall_x && d->ny >= 8 && d->nx % (d->storage == kFP32 ? 4 : 8) == 0;
}

cudaError_t launch_step_mode(const pflbm_domain* d, int mode, const StepArgs& a) {
  const int form = d->par.force;
  switch (d->storage) {
    case kFP32: return launch_step_fp32(form, mode, a, d->stream);
    case kFP16: return launch_step_fp16(form, mode, a, d->stream);
    default: return launch_step_bf16(form, mode, a, d->stream);
  }
}

cudaError_t launch_step(const pflbm_domain* d, const StepArgs& a) {
  return launch_step_mode(d, d->mode, a);
}

void drop_graph(pflbm_domain* d) {
  if (d->gexec) cudaGraphExecDestroy(d->gexec);
  d->gexec = nullptr;
}

// One plain step from the current buffer.
pflbm_status plain_step(pflbm_domain* d) {
  StepArgs a = make_args(d, d->cur);
  a.first = d->t == 0;
  a.macro = 0;
  cudaError_t e = launch_step(d, a);
  if (e != cudaSuccess) {
    set_err("step launch", e);
    return PFLBM_ECUDA;
  }
  d->cur = 1 - d->cur;
  d->t += 1;
  return PFLBM_OK;
}

// Capture kGraphSteps steps (buffers alternating from the current parity).
pflbm_status capture_graph(pflbm_domain* d) {
  drop_graph(d);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(d->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    set_err("graph capture", e);
    return PFLBM_ECUDA;
  }
  int from = d->cur;
  for (int k = 0; k < kGraphSteps; ++k) {
    StepArgs a = make_args(d, from);
    a.first = 0;
    a.macro = 0;
    e = launch_step(d, a);
    if (e != cudaSuccess) break;
    from = 1 - from;
  }
  cudaError_t e2 = cudaStreamEndCapture(d->stream, &g);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&d->gexec, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    d->gexec = nullptr;
    set_err("graph instantiate", e);
    return PFLBM_ECUDA;
  }
  d->g_parity = d->cur;
  return PFLBM_OK;
}

// Macroscopic fields of the current state into the staging buffer.
pflbm_status stage_fields(pflbm_domain* d) {
  StepArgs a = make_args(d, d->cur);
  a.first = d->t == 0;
  a.macro = 1;
  cudaError_t e = launch_step(d, a);
  if (e != cudaSuccess) {
    set_err("field pass", e);
    return PFLBM_ECUDA;
  }
  return PFLBM_OK;
}

pflbm_status copy_out(pflbm_domain* d, void* dst, const void* src, size_t bytes, int on_device) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  d->stream);
  if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(d->stream);
  if (e != cudaSuccess) {
    set_err("copy", e);
    return PFLBM_ECUDA;
  }
  return PFLBM_OK;
}

}  // namespace

extern "C" {

size_t pflbm_workspace_bytes(int nx, int ny, pflbm_storage storage) {
  Layout L;
  if (!layout_of(nx, ny, (int)storage, &L)) return 0;
  return L.total;
}

pflbm_status pflbm_create(int nx, int ny, pflbm_bc bc_x, pflbm_bc bc_y, pflbm_storage storage,
                          void* dev_workspace, size_t ws_bytes, void* cuda_stream,
                          pflbm_domain** out) {
  if (!out) return PFLBM_EINVAL;
  *out = nullptr;
  Layout L;
  if ((bc_x != PFLBM_PERIODIC && bc_x != PFLBM_FREESLIP) ||
      (bc_y != PFLBM_PERIODIC && bc_y != PFLBM_WALL) ||
      !layout_of(nx, ny, (int)storage, &L) || !dev_workspace ||
      ((uintptr_t)dev_workspace % kAlign) != 0) {
    set_msg("pflbm_create: invalid argument");
    return PFLBM_EINVAL;
  }
  if (ws_bytes < L.total) {
    set_msg("pflbm_create: workspace too small");
    return PFLBM_ENOMEM_WS;
  }
  pflbm_domain* d = new (std::nothrow) pflbm_domain;
  if (!d) return PFLBM_EINVAL;
  memset(d, 0, sizeof(*d));
  d->nx = nx;
  d->ny = ny;
  d->wall = bc_y == PFLBM_WALL;
  d->wall_x = bc_x == PFLBM_FREESLIP;
  d->storage = (int)storage;
  d->stream = (cudaStream_t)cuda_stream;
  d->ws = (char*)dev_workspace;
  d->lay = L;
  d->mode = kGather;
  *out = d;
  return PFLBM_OK;
}

pflbm_status pflbm_set_params(pflbm_domain* d, const pflbm_params* p) {
  if (!d || !p) return PFLBM_EINVAL;
  const bool ok = p->sigma >= 0 && p->W > 0 && p->M > 0 && p->tau_h > 0.5 && p->rho1 > 0 &&
                  p->rho2 > 0 && p->nu1 > 0 && p->nu2 > 0 && p->eps >= 0 && p->force >= 0 &&
                  p->force <= 7 && isfinite(p->gx) && isfinite(p->gy) &&
                  isfinite(p->uw_bottom) && isfinite(p->uw_top) && isfinite(p->sigma) &&
                  (p->scale_f == 0 || is_pow2(p->scale_f)) &&
                  (p->scale_h == 0 || is_pow2(p->scale_h));
  if (!ok) {
    set_msg("pflbm_set_params: parameter out of range");
    return PFLBM_EINVAL;
  }
  if (d->wall_x && (p->gx != 0 || p->uw_bottom != 0 || p->uw_top != 0)) {
    set_msg("pflbm_set_params: free-slip side walls need gx = 0 and walls at rest in y");
    return PFLBM_EINVAL;
  }
  d->par = *p;
  const double beta = 0.75 * p->sigma / p->W, kappa = 0.375 * p->W * p->sigma;
  const double th = p->tau_h;
  Phys& q = d->phys;
  q.beta4 = (float)(4 * beta);
  q.kappa = (float)kappa;
  q.half_sigma = (float)(0.5 * p->sigma);
  q.eps2 = (float)(p->eps * p->eps);
  q.rho_mid = (float)(0.5 * (p->rho1 + p->rho2));
  q.drho_half = (float)(0.5 * (p->rho1 - p->rho2));
  q.mu_mid = (float)(0.5 * (p->rho1 * p->nu1 + p->rho2 * p->nu2));
  q.mu_dhalf = (float)(0.5 * (p->rho1 * p->nu1 - p->rho2 * p->nu2));
  q.gx = (float)p->gx;
  q.gy = (float)p->gy;
  q.rho0 = isnan(p->rho0) ? q.rho_mid : (float)p->rho0;  // refined at init
  if (isnan(p->rho0) && d->has_mean_phi0) q.rho0 = default_rho0(d);
  q.uwb = (float)p->uw_bottom;
  q.uwt = (float)p->uw_top;
  q.inv_tau_h = (float)(1.0 / th);
  q.hforce = (float)(1.0 - 0.5 / th);
  q.eta = (float)(p->M / ((th - 0.5) / 3.0));
  q.acoef = (float)(3.0 * (th * th - th + 1.0 / 6.0) / (th * (th - 0.5)));
  double s_auto = 1.0;
  if (p->sigma > 0) s_auto = exp2(round(log2(4.0 / p->sigma)));
  const double sf = p->scale_f > 0 ? p->scale_f : s_auto;
  const double sh = p->scale_h > 0 ? p->scale_h : s_auto;
  q.sf = (float)sf;
  q.inv_sf = (float)(1.0 / sf);
  q.sh = (float)sh;
  q.inv_sh = (float)(1.0 / sh);
  d->has_params = 1;
  drop_graph(d);
  return PFLBM_OK;
}

pflbm_status pflbm_init_phi(pflbm_domain* d, const float* phi0, int on_device) {
  if (!d || !phi0) return PFLBM_EINVAL;
  if (!d->has_params) {
    set_msg("pflbm_init_phi: parameters not set");
    return PFLBM_ESTATE;
  }
  const size_t n = (size_t)d->nx * d->ny;
  float* stage = reinterpret_cast<float*>(d->ws + d->lay.fields);
  cudaError_t e = cudaMemcpyAsync(stage, phi0, n * 4,
                                  on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                  d->stream);
  // zero both population buffers (ghost rows included)
  if (e == cudaSuccess) e = cudaMemsetAsync(d->ws, 0, d->lay.phiu, d->stream);
  d->cur = 0;
  StepArgs a = make_args(d, 1);  // writes go to buffer 0
  if (e == cudaSuccess) e = launch_init(d->storage, a, stage, d->stream);
  if (e != cudaSuccess) {
    set_err("init", e);
    return PFLBM_ECUDA;
  }
  if (isnan(d->par.rho0)) {
    // rho is linear in phi, so the mean density is rho(mean phi0)
    Lattice L = a.L;
    DiagGeom g = {0, 0, 0, 0, 0};
    double* red = reinterpret_cast<double*>(d->ws + d->lay.red);
    double* part = reinterpret_cast<double*>(d->ws + d->lay.partials);
    // the diagnostics read phi from field slot 0, which holds phi0 here;
    // the other slots are not needed for the sum of phi
    e = cudaMemsetAsync(stage + n, 0, (kNFields - 1) * n * 4, d->stream);
    if (e == cudaSuccess) e = launch_diag(L, stage, g, part, kMaxDiagBlocks, red, d->stream);
    double h[kNRed];
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h, red, sizeof(h), cudaMemcpyDeviceToHost, d->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
    if (e != cudaSuccess) {
      set_err("init mean density", e);
      return PFLBM_ECUDA;
    }
    d->mean_phi0 = h[0] / (double)n;
    d->has_mean_phi0 = 1;
    d->phys.rho0 = default_rho0(d);
  } else {
    d->has_mean_phi0 = 0;
  }
  e = cudaMemsetAsync(d->ws + d->lay.err, 0, 4, d->stream);
  if (e != cudaSuccess) {
    set_err("init", e);
    return PFLBM_ECUDA;
  }
  build_maps(d);
  d->t = 0;
  d->has_state = 1;
  drop_graph(d);
  return PFLBM_OK;
}

pflbm_status pflbm_set_stage_mode(pflbm_domain* d, int mode) {
  if (!d || mode < 0 || mode >= kNumModes) return PFLBM_EINVAL;
  if (d->wall_x && mode != kGather && mode != kGather8) {
    set_msg("pflbm_set_stage_mode: side walls are staged by gathers only");
    return PFLBM_EINVAL;
  }
  if (mode == kMarch && !march_ok(d)) {
    set_msg("pflbm_set_stage_mode: the march needs nx a multiple of 4 (float32) or 8 "
            "(16-bit storage) and ny >= 8");
    return PFLBM_EINVAL;
  }
  d->mode = mode;
  drop_graph(d);
  return PFLBM_OK;
}

int pflbm_get_stage_mode(const pflbm_domain* d) { return d ? d->mode : -1; }

pflbm_status pflbm_autotune(pflbm_domain* d, int trial_steps, int* mode_out) {
  if (!d || trial_steps < 1) return PFLBM_EINVAL;
  if (!d->has_state) {
    set_msg("pflbm_autotune: no initial state");
    return PFLBM_ESTATE;
  }
  // Trial steps read the current buffer and write the spare one without
  // flipping buffers or writing (phi u) back, so the state is unchanged.
  StepArgs a = make_args(d, d->cur);
  a.first = d->t == 0;
  a.macro = 0;
  a.keep_phiu = 1;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 1e30f;
  int best_mode = d->mode;
  for (int m = 0; m < kNumModes && e == cudaSuccess; ++m) {
    if (d->wall_x && m != kGather && m != kGather8) continue;  // side walls: gathers only
    if (m == kMarch && !march_ok(d)) continue;
    e = launch_step_mode(d, m, a);  // warm-up (also sets kernel attributes)
    if (e == cudaSuccess) e = cudaEventRecord(e0, d->stream);
    for (int k = 0; k < trial_steps && e == cudaSuccess; ++k) e = launch_step_mode(d, m, a);
    if (e == cudaSuccess) e = cudaEventRecord(e1, d->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && ms < best) {
      best = ms;
      best_mode = m;
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    set_err("autotune", e);
    return PFLBM_ECUDA;
  }
  d->mode = best_mode;
  drop_graph(d);
  if (mode_out) *mode_out = best_mode;
  return PFLBM_OK;
}

pflbm_status pflbm_set_tma(pflbm_domain* d, int enable) {
  if (!d) return PFLBM_EINVAL;
  d->tma_off = enable ? 0 : 1;
  drop_graph(d);
  return PFLBM_OK;
}

pflbm_status pflbm_set_graphs(pflbm_domain* d, int enable) {
  if (!d) return PFLBM_EINVAL;
  if (enable && d->stream == nullptr) {
    set_msg("pflbm_set_graphs: graphs need a non-default stream");
    return PFLBM_EINVAL;
  }
  d->graphs = enable != 0;
  if (!d->graphs) drop_graph(d);
  return PFLBM_OK;
}

pflbm_status pflbm_step(pflbm_domain* d, int nsteps) {
  if (!d || nsteps < 0) return PFLBM_EINVAL;
  if (!d->has_state) {
    set_msg("pflbm_step: no initial state");
    return PFLBM_ESTATE;
  }
  pflbm_status st = PFLBM_OK;
  int left = nsteps;
  while (left > 0 && d->t == 0) {
    if ((st = plain_step(d)) != PFLBM_OK) return st;
    --left;
  }
  if (d->graphs && left >= kGraphSteps) {
    if (!d->gexec || d->g_parity != d->cur) {
      if (d->gexec && d->g_parity != d->cur) {
        if ((st = plain_step(d)) != PFLBM_OK) return st;
        --left;
      }
      if (!d->gexec && (st = capture_graph(d)) != PFLBM_OK) return st;
    }
    while (left >= kGraphSteps) {
      cudaError_t e = cudaGraphLaunch(d->gexec, d->stream);
      if (e != cudaSuccess) {
        set_err("graph launch", e);
        return PFLBM_ECUDA;
      }
      d->t += kGraphSteps;  // even: parity unchanged
      left -= kGraphSteps;
    }
  }
  while (left-- > 0)
    if ((st = plain_step(d)) != PFLBM_OK) return st;
  return PFLBM_OK;
}

long long pflbm_steps_done(const pflbm_domain* d) { return d ? d->t : -1; }

pflbm_status pflbm_read_fields(pflbm_domain* d, float* dst, int on_device) {
  if (!d || !dst) return PFLBM_EINVAL;
  if (!d->has_state) return PFLBM_ESTATE;
  pflbm_status st = stage_fields(d);
  if (st != PFLBM_OK) return st;
  const size_t n = (size_t)d->nx * d->ny;
  return copy_out(d, dst, d->ws + d->lay.fields, (size_t)kNFields * n * 4, on_device);
}

pflbm_status pflbm_read(pflbm_domain* d, pflbm_field field, float* dst, int on_device) {
  if (!d || !dst || (int)field < 0 || (int)field >= kNFields) return PFLBM_EINVAL;
  if (!d->has_state) return PFLBM_ESTATE;
  pflbm_status st = stage_fields(d);
  if (st != PFLBM_OK) return st;
  const size_t n = (size_t)d->nx * d->ny;
  return copy_out(d, dst, d->ws + d->lay.fields + (size_t)field * n * 4, n * 4, on_device);
}

pflbm_status pflbm_read_populations(pflbm_domain* d, float* f_out, float* h_out, int on_device) {
  if (!d || (!f_out && !h_out)) return PFLBM_EINVAL;
  if (!d->has_state) return PFLBM_ESTATE;
  const size_t n = (size_t)d->nx * d->ny;
  // stage through the field buffer (9 fields of n floats fit 9 populations)
  float* stage = reinterpret_cast<float*>(d->ws + d->lay.fields);
  StepArgs a = make_args(d, d->cur);
  float* outs[2] = {f_out, h_out};
  for (int w = 0; w < 2; ++w) {
    if (!outs[w]) continue;
    cudaError_t e = launch_read_pops(d->storage, a, w == 0 ? stage : nullptr,
                                     w == 1 ? stage : nullptr, d->stream);
    if (e != cudaSuccess) {
      set_err("read populations", e);
      return PFLBM_ECUDA;
    }
    pflbm_status st = copy_out(d, outs[w], stage, 9 * n * 4, on_device);
    if (st != PFLBM_OK) return st;
  }
  return PFLBM_OK;
}

pflbm_status pflbm_diagnostics(pflbm_domain* d, const pflbm_diag_geom* geom, pflbm_diag* out) {
  if (!d || !out) return PFLBM_EINVAL;
  if (!d->has_state) return PFLBM_ESTATE;
  pflbm_status st = stage_fields(d);
  if (st != PFLBM_OK) return st;
  DiagGeom g = {0, 0, 0, 0, 0};
  if (geom) g = DiagGeom{geom->xc, geom->yc, geom->r_in, geom->r_out, 1};
  StepArgs a = make_args(d, d->cur);
  double* red = reinterpret_cast<double*>(d->ws + d->lay.red);
  double* part = reinterpret_cast<double*>(d->ws + d->lay.partials);
  cudaError_t e = launch_diag(a.L, a.fields, g, part, kMaxDiagBlocks, red, d->stream);
  double h[kNRed];
  int err_word = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, red, sizeof(h), cudaMemcpyDeviceToHost, d->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&err_word, d->ws + d->lay.err, 4, cudaMemcpyDeviceToHost, d->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
  if (e != cudaSuccess) {
    set_err("diagnostics", e);
    return PFLBM_ECUDA;
  }
  memset(out, 0, sizeof(*out));
  out->mass = h[0];
  out->umax = sqrt(h[1]);
  out->area1 = h[2];
  out->R_num = sqrt(h[2] / M_PI);
  if (g.has_geom && h[9] > 0 && h[11] > 0) {
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
  if (err_word) {
    set_msg("a bounded device wait expired during a step");
    return PFLBM_ETIMEOUT;
  }
  return h[12] > 0 ? PFLBM_EUNSTABLE : PFLBM_OK;
}

pflbm_status pflbm_bubble_diagnostics(pflbm_domain* d, pflbm_bubble_diag* out) {
  if (!d || !out) return PFLBM_EINVAL;
  if (!d->has_state) return PFLBM_ESTATE;
  pflbm_status st = stage_fields(d);
  if (st != PFLBM_OK) return st;
  StepArgs a = make_args(d, d->cur);
  double* red = reinterpret_cast<double*>(d->ws + d->lay.red);
  double* part = reinterpret_cast<double*>(d->ws + d->lay.partials);
  cudaError_t e = launch_bubble_diag(a.L, a.fields, part, kMaxDiagBlocks, red, d->stream);
  double h[kNRed];
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, red, sizeof(h), cudaMemcpyDeviceToHost, d->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
  if (e != cudaSuccess) {
    set_err("bubble diagnostics", e);
    return PFLBM_ECUDA;
  }
  memset(out, 0, sizeof(*out));
  out->mass2 = h[0];
  if (h[0] > 0) {
    out->xc2 = h[1] / h[0];
    out->yc2 = h[2] / h[0];
    out->uc2 = h[3] / h[0];
    out->vc2 = h[4] / h[0];
  }
  out->area2 = h[5];
  out->perimeter = h[6];
  out->circularity = h[6] > 0 ? 2.0 * sqrt(M_PI * h[5]) / h[6] : 0.0;
  out->nonfinite = h[7];
  return h[7] > 0 ? PFLBM_EUNSTABLE : PFLBM_OK;
}

size_t pflbm_state_bytes(const pflbm_domain* d) {
  if (!d) return 0;
  // header (step count, magic) + the current population buffers + phi u
  const Layout& L = d->lay;
  return 64 + (L.h[0] - L.f[0]) + (L.h0[0] - L.h[0]) + (L.f[1] - L.h0[0]) + (L.fields - L.phiu);
}

pflbm_status pflbm_save_state(pflbm_domain* d, void* dst, int on_device) {
  if (!d || !dst) return PFLBM_EINVAL;
  if (!d->has_state) return PFLBM_ESTATE;
  const Layout& L = d->lay;
  // header: magic, step, nx, ny, storage, walls y and x, and (second magic)
  // the bits of mean phi0 that the default rho0 of the run follows from
  long long hdr[8] = {d->has_mean_phi0 ? kStateMagicMean : kStateMagic, d->t, d->nx, d->ny,
                      d->storage, d->wall, d->wall_x, 0};
  if (d->has_mean_phi0) memcpy(&hdr[7], &d->mean_phi0, sizeof(double));
  char* p = (char*)dst;
  const cudaMemcpyKind h2x = on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
  const cudaMemcpyKind d2x = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  cudaError_t e = cudaMemcpyAsync(p, hdr, sizeof(hdr), h2x, d->stream);
  p += 64;
  const int c = d->cur;
  const size_t sz_f = L.h[0] - L.f[0], sz_h = L.h0[0] - L.h[0], sz_h0 = L.f[1] - L.h0[0];
  if (e == cudaSuccess) e = cudaMemcpyAsync(p, d->ws + L.f[c], sz_f, d2x, d->stream);
  p += sz_f;
  if (e == cudaSuccess) e = cudaMemcpyAsync(p, d->ws + L.h[c], sz_h, d2x, d->stream);
  p += sz_h;
  if (sz_h0 && e == cudaSuccess) e = cudaMemcpyAsync(p, d->ws + L.h0[c], sz_h0, d2x, d->stream);
  p += sz_h0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(p, d->ws + L.phiu, L.fields - L.phiu, d2x, d->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
  if (e != cudaSuccess) {
    set_err("save_state", e);
    return PFLBM_ECUDA;
  }
  return PFLBM_OK;
}

pflbm_status pflbm_load_state(pflbm_domain* d, const void* src, int on_device) {
  if (!d || !src) return PFLBM_EINVAL;
  if (!d->has_params) return PFLBM_ESTATE;
  const Layout& L = d->lay;
  long long hdr[8];
  cudaError_t e = cudaMemcpyAsync(hdr, src, sizeof(hdr),
                                  on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost,
                                  d->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
  if (e != cudaSuccess) {
    set_err("load_state", e);
    return PFLBM_ECUDA;
  }
  if ((hdr[0] != kStateMagic && hdr[0] != kStateMagicMean) || hdr[2] != d->nx ||
      hdr[3] != d->ny || hdr[4] != d->storage || hdr[5] != d->wall || hdr[6] != d->wall_x) {
    set_msg("pflbm_load_state: state does not match this domain");
    return PFLBM_EINVAL;
  }
  const char* p = (const char*)src + 64;
  const cudaMemcpyKind x2d = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const size_t sz_f = L.h[0] - L.f[0], sz_h = L.h0[0] - L.h[0], sz_h0 = L.f[1] - L.h0[0];
  d->cur = 0;
  e = cudaMemcpyAsync(d->ws + L.f[0], p, sz_f, x2d, d->stream);
  p += sz_f;
  if (e == cudaSuccess) e = cudaMemcpyAsync(d->ws + L.h[0], p, sz_h, x2d, d->stream);
  p += sz_h;
  if (sz_h0 && e == cudaSuccess) e = cudaMemcpyAsync(d->ws + L.h0[0], p, sz_h0, x2d, d->stream);
  p += sz_h0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(d->ws + L.phiu, p, L.fields - L.phiu, x2d, d->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
  if (e != cudaSuccess) {
    set_err("load_state", e);
    return PFLBM_ECUDA;
  }
  e = cudaMemsetAsync(d->ws + L.err, 0, 4, d->stream);
  if (e != cudaSuccess) {
    set_err("load_state", e);
    return PFLBM_ECUDA;
  }
  build_maps(d);
  d->t = hdr[1];
  d->has_state = 1;
  d->has_mean_phi0 = hdr[0] == kStateMagicMean;
  if (d->has_mean_phi0) {
    memcpy(&d->mean_phi0, &hdr[7], sizeof(double));
    if (isnan(d->par.rho0)) d->phys.rho0 = default_rho0(d);
  }
  drop_graph(d);
  return PFLBM_OK;
}

void pflbm_destroy(pflbm_domain* d) {
  if (!d) return;
  drop_graph(d);
  delete d;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// adjoint with checkpointing
// ---------------------------------------------------------------------------
namespace {

struct AdjLayout {
  // tape[1]: a second tape, so that the recomputation of the segment before
  // can run while a segment is reversed (two segments or more)
  size_t ckpt, tape[2], work, adj[2], acc, final_state, total;
  size_t blob;       // bytes of one state blob
  size_t tape_step;  // bytes of one step's tape
  int ncp;
};

bool adj_layout(const pflbm_domain* d, int nsteps, int every, AdjLayout* L) {
  if (!d || nsteps < 1 || every < 1 || d->storage != kFP32 || d->wall_x) return false;
  const size_t n = (size_t)d->nx * d->ny;
  // the taping step addresses its planes with 32-bit offsets
  if ((size_t)kTapePlanes * n >= ((size_t)1 << 31)) return false;
  L->blob = align_up(pflbm_state_bytes(d));
  L->ncp = (nsteps + every - 1) / every;
  size_t off = 0;
  L->ckpt = off;  // the start of every segment but the last (taped in the forward run)
  off += (size_t)(L->ncp - 1) * L->blob;
  L->final_state = off;
  off += L->blob;
  L->tape_step = align_up((size_t)kTapePlanes * n * 4);
  const size_t seg_tape = (size_t)(every < nsteps ? every : nsteps) * L->tape_step;
  L->tape[0] = off;  // one tape per step of a segment
  off += seg_tape;
  L->tape[1] = L->tape[0];
  if (L->ncp > 1) {
    L->tape[1] = off;
    off += seg_tape;
  }
  L->work = off;
  off = align_up(off + (size_t)kWorkPlanes * n * 4);
  for (int b = 0; b < 2; ++b) {
    L->adj[b] = off;
    off = align_up(off + (size_t)(kAdjScalar + kAdjPlanes) * n * 4);
  }
  L->acc = off;
  off = align_up(off + 4 * sizeof(double));
  L->total = off;
  return true;
}

// Graphs of one adjoint run: the recomputation of a segment keyed by (first
// segment, full length) and its reverse sweep keyed by (first segment, parity
// of the adjoint buffers, full length).
struct AdjGraphs {
  cudaGraphExec_t rec[2][2][2] = {};     // [first][full][tape]
  cudaGraphExec_t rev[2][2][2][2] = {};  // [first][parity][full][tape]
  ~AdjGraphs() {
    for (auto& a : rec)
      for (auto& b : a)
        for (auto& g : b)
          if (g) cudaGraphExecDestroy(g);
    for (auto& a : rev)
      for (auto& b : a)
        for (auto& c : b)
          for (auto& g : c)
            if (g) cudaGraphExecDestroy(g);
  }
};

// Streams and events of the reverse sweep: the recomputation of segment c - 1
// (checkpoint load and taping steps, on the auxiliary stream) runs while
// segment c is reversed on the domain's stream.
struct AdjOverlap {
  cudaStream_t aux = nullptr;
  cudaEvent_t fwd = nullptr, rec = nullptr, rev[2] = {nullptr, nullptr};
  cudaError_t create() {
    cudaError_t e = cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fwd, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&rec, cudaEventDisableTiming);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k)
      e = cudaEventCreateWithFlags(&rev[k], cudaEventDisableTiming);
    return e;
  }
  ~AdjOverlap() {
    if (aux) cudaStreamSynchronize(aux);
    for (cudaEvent_t ev : {fwd, rec, rev[0], rev[1]})
      if (ev) cudaEventDestroy(ev);
    if (aux) cudaStreamDestroy(aux);
  }
};

// Run a sequence of launches on stream s from the graph in *cache, capturing
// and instantiating it on first use; on a stream that cannot be captured (the
// legacy default stream) the launches run directly.
template <class Fn>
cudaError_t run_captured(cudaStream_t s, cudaGraphExec_t* cache, Fn&& launches) {
  if (*cache) return cudaGraphLaunch(*cache, s);
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return launches();
  }
  const cudaError_t el = launches();
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(s, &g);
  if (el != cudaSuccess) e = el;
  if (e == cudaSuccess) e = cudaGraphInstantiate(cache, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    *cache = nullptr;
    return e;
  }
  return cudaGraphLaunch(*cache, s);
}

}  // namespace

extern "C" {

size_t pflbm_adjoint_scratch_bytes(const pflbm_domain* d, int nsteps, int ckpt_every) {
  AdjLayout L;
  return adj_layout(d, nsteps, ckpt_every, &L) ? L.total : 0;
}

pflbm_status pflbm_adjoint_run(pflbm_domain* d, const float* phi0, int nsteps, int ckpt_every,
                               const float* dJ_dphiT, float* dJ_dphi0, double* dJ_dsigma,
                               double* dJ_dM, void* scratch, size_t scratch_bytes) {
  AdjLayout L;
  if (!d || !phi0 || !dJ_dphiT || !dJ_dphi0 || !scratch ||
      !adj_layout(d, nsteps, ckpt_every, &L)) {
    set_msg("pflbm_adjoint_run: invalid argument (FP32 storage, periodic x, nsteps, "
            "ckpt_every >= 1)");
    return PFLBM_EINVAL;
  }
  if (!d->has_params) return PFLBM_ESTATE;
  if (scratch_bytes < L.total || ((uintptr_t)scratch % kAlign) != 0) {
    set_msg("pflbm_adjoint_run: scratch too small or misaligned");
    return PFLBM_ENOMEM_WS;
  }
  char* S = (char*)scratch;
  const size_t n = (size_t)d->nx * d->ny;
  pflbm_status st;
  cudaError_t e = cudaSuccess;
  auto fail = [&](const char* what) {
    set_err(what, e);
    return PFLBM_ECUDA;
  };
  // forward with a checkpoint every ckpt_every steps and the final state; the
  // last segment is taped on the way, so its reverse needs no recomputation
  if ((e = setup_tape_step(d->par.force)) != cudaSuccess) return fail("adjoint set-up");
  if ((st = pflbm_init_phi(d, phi0, 1)) != PFLBM_OK) return st;
  for (int c = 0; c < L.ncp; ++c) {
    const int seg = c + 1 < L.ncp ? ckpt_every : nsteps - c * ckpt_every;
    if (c + 1 < L.ncp) {
      if ((st = pflbm_save_state(d, S + L.ckpt + (size_t)c * L.blob, 1)) != PFLBM_OK) return st;
      if ((st = pflbm_step(d, seg)) != PFLBM_OK) return st;
      continue;
    }
    for (int j = 0; j < seg; ++j) {
      StepArgs a = make_args(d, d->cur);
      a.first = d->t == 0;
      a.tape = reinterpret_cast<float*>(S + L.tape[0] + (size_t)j * L.tape_step);
      if ((e = launch_tape_step(d->par.force, a, d->stream)) != cudaSuccess)
        return fail("adjoint forward");
      d->cur = 1 - d->cur;
      d->t += 1;
    }
  }
  if ((st = pflbm_save_state(d, S + L.final_state, 1)) != PFLBM_OK) return st;

  // adjoint of the final state: dJ/dh_i = dJ/dphi_T for every i (the per-node
  // scalar of h), f and q zero
  int cur = 0;
  float* adj[2] = {reinterpret_cast<float*>(S + L.adj[0]), reinterpret_cast<float*>(S + L.adj[1])};
  double* acc = reinterpret_cast<double*>(S + L.acc);
  e = cudaMemsetAsync(adj[0], 0, (size_t)(kAdjScalar + kAdjPlanes) * n * 4, d->stream);
  if (e == cudaSuccess)  // dJ/dphi_T into the PHI (4th) float of each node's scalar block
    e = cudaMemcpy2DAsync(adj[0] + 3, 4 * sizeof(float), dJ_dphiT, sizeof(float), sizeof(float),
                          n, cudaMemcpyDeviceToDevice, d->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, 4 * sizeof(double), d->stream);
  if (e != cudaSuccess) return fail("adjoint setup");

  AdjArgs A;
  memset(&A, 0, sizeof(A));
  A.g = AdjGeo{d->nx, d->ny, d->wall};
  A.p = d->phys;
  A.form = d->par.force;
  A.W = reinterpret_cast<float*>(S + L.work);
  A.acc = acc;
  AdjGraphs graphs;
  AdjOverlap ov;
  if (L.ncp > 1) {
    if ((e = ov.create()) != cudaSuccess) return fail("adjoint streams");
    if ((e = cudaEventRecord(ov.fwd, d->stream)) != cudaSuccess) return fail("adjoint streams");
  }
  // segment c reads the tape its recomputation wrote: the last segment the
  // one the forward run taped, then the two tapes alternate
  const auto tape_index = [&](int c) { return (L.ncp - 1 - c) & 1; };
  // Recompute segment c (never the last) from its checkpoint on the auxiliary
  // stream, taping every step, and mark its end with ov.rec.
  const auto recompute = [&](int c) -> pflbm_status {
    const int first = c == 0, tb = tape_index(c);
    cudaStream_t keep = d->stream;
    d->stream = ov.aux;  // the checkpoint load runs on the auxiliary stream too
    pflbm_status st2 = pflbm_load_state(d, S + L.ckpt + (size_t)c * L.blob, 1);
    if (st2 == PFLBM_OK) {
      e = run_captured(ov.aux, &graphs.rec[first][1][tb], [&]() -> cudaError_t {
        for (int j = 0; j < ckpt_every; ++j) {
          StepArgs a = make_args(d, j & 1);
          a.first = first && j == 0;
          a.tape = reinterpret_cast<float*>(S + L.tape[tb] + (size_t)j * L.tape_step);
          const cudaError_t el = launch_tape_step(d->par.force, a, ov.aux);
          if (el != cudaSuccess) return el;
        }
        return cudaSuccess;
      });
      if (e == cudaSuccess) e = cudaEventRecord(ov.rec, ov.aux);
      if (e != cudaSuccess) st2 = fail("adjoint recompute");
    }
    d->stream = keep;
    return st2;
  };
  for (int c = L.ncp - 1; c >= 0; --c) {
    const int seg = c + 1 < L.ncp ? ckpt_every : nsteps - c * ckpt_every;
    const int first = c == 0, full = seg == ckpt_every, tb = tape_index(c);
    // the recomputation of this segment (the last one was taped by the forward
    // run) has finished before its reverse starts
    if (c + 1 < L.ncp && (e = cudaStreamWaitEvent(d->stream, ov.rec, 0)) != cudaSuccess)
      return fail("adjoint streams");
    // reverse through the segment
    const int cur0 = cur;
    e = run_captured(d->stream, &graphs.rev[first][cur0][full][tb], [&]() -> cudaError_t {
      int cc = cur0;
      for (int j = seg - 1; j >= 0; --j) {
        A.tape = reinterpret_cast<const float*>(S + L.tape[tb] + (size_t)j * L.tape_step);
        A.first = first && j == 0;
        A.ain = adj[cc];
        A.aout = adj[1 - cc];
        const cudaError_t el = launch_adjoint_step(A, d->stream);
        if (el != cudaSuccess) return el;
        cc = 1 - cc;
      }
      return cudaSuccess;
    });
    if (e != cudaSuccess) return fail("adjoint step");
    cur = (seg & 1) ? 1 - cur0 : cur0;
    if (L.ncp > 1 && (e = cudaEventRecord(ov.rev[c & 1], d->stream)) != cudaSuccess)
      return fail("adjoint streams");
    // meanwhile the segment before is recomputed into the tape that the
    // segment after this one was reversed from (or, first, the unused one)
    if (c >= 1) {
      const cudaEvent_t free_tape = c + 1 < L.ncp ? ov.rev[(c + 1) & 1] : ov.fwd;
      if ((e = cudaStreamWaitEvent(ov.aux, free_tape, 0)) != cudaSuccess)
        return fail("adjoint streams");
      if ((st = recompute(c - 1)) != PFLBM_OK) return st;
    }
  }
  // through the initial state to phi0
  A.ain = adj[cur];
  if ((e = launch_adjoint_init(A, phi0, dJ_dphi0, d->stream)) != cudaSuccess)
    return fail("adjoint init");
  double h[4];
  e = cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, d->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(d->stream);
  if (e != cudaSuccess) return fail("adjoint gradients");
  // beta4 = 3 sigma / W, kappa = 3 W sigma / 8, eta = M / (cs^2 (tau_h - 1/2))
  const double W = d->par.W;
  if (dJ_dsigma) *dJ_dsigma = h[0] * 3.0 / W + h[1] * 3.0 * W / 8.0 + h[3];
  if (dJ_dM) *dJ_dM = h[2] * 3.0 / (d->par.tau_h - 0.5);
  // leave the domain at the final state of the forward run
  return pflbm_load_state(d, S + L.final_state, 1);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// batch
// ---------------------------------------------------------------------------
struct pflbm_batch {
  int n;
  pflbm_domain** doms;
  cudaStream_t stream;
  char* ws;
  size_t table_off;
  // work-lists for tiles of kTY rows ([0]) and of kShortRows rows ([1])
  size_t items_off[2];
  size_t tickets_off;  // the batch kernel's item counter
  int nitems[2];
  int mode, ctas_per_sm, rows;
  int graphs;
  cudaGraphExec_t gexec;
  StepArgs* host_table;  // staging of the argument table
};

namespace {

constexpr int kBatchGraphSteps = 16;  // steps captured per batch graph (even)

long long tiles_of(const pflbm_domain* d, int rows) {
  return (long long)((d->nx + kTX - 1) / kTX) * ((d->ny + rows - 1) / rows);
}
int rows_slot(int rows) { return rows == kTY ? 0 : 1; }
constexpr int kBatchRows[2] = {kTY, kShortRows};

void batch_drop_graph(pflbm_batch* b) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  b->gexec = nullptr;
}

// Upload the argument table from the domains' current states: entry 2 i + p
// steps domain i from buffer cur_i ^ p; with `firsts`, domains at t = 0 get
// the first-step flag.
cudaError_t upload_table(pflbm_batch* b, int keep_phiu, int firsts) {
  for (int i = 0; i < b->n; ++i) {
    for (int p = 0; p < 2; ++p) {
      StepArgs a = make_args(b->doms[i], b->doms[i]->cur ^ p);
      a.first = firsts && b->doms[i]->t == 0;
      a.macro = 0;
      a.keep_phiu = keep_phiu;
      b->host_table[2 * i + p] = a;
    }
  }
  cudaError_t e = cudaMemcpyAsync(b->ws + b->table_off, b->host_table,
                                  sizeof(StepArgs) * 2 * b->n, cudaMemcpyHostToDevice, b->stream);
  // the host table is reused by the next upload: wait for this copy
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return e;
}

int batch_grid(const pflbm_batch* b) {
  const long long g = (long long)num_sms() * b->ctas_per_sm;
  const int n = b->nitems[rows_slot(b->rows)];
  return (int)(g < n ? g : n);
}

cudaError_t batch_launch(const pflbm_batch* b, int bp) {
  const int r = rows_slot(b->rows);
  return launch_batch(b->mode, b->rows, reinterpret_cast<const StepArgs*>(b->ws + b->table_off),
                      reinterpret_cast<const int4*>(b->ws + b->items_off[r]), b->nitems[r], bp,
                      batch_grid(b), reinterpret_cast<unsigned*>(b->ws + b->tickets_off),
                      b->stream);
}

}  // namespace

extern "C" {

size_t pflbm_batch_workspace_bytes(int n, pflbm_domain* const* doms) {
  if (n <= 0 || !doms) return 0;
  size_t bytes = align_up(sizeof(StepArgs) * 2 * (size_t)n);
  for (int r = 0; r < 2; ++r) {
    long long items = 0;
    for (int i = 0; i < n; ++i) {
      if (!doms[i]) return 0;
      items += tiles_of(doms[i], kBatchRows[r]);
    }
    bytes += align_up(sizeof(int4) * (size_t)items);
  }
  return bytes + align_up(sizeof(unsigned));  // the item counter
}

pflbm_status pflbm_batch_create(int n, pflbm_domain* const* doms, void* dev_workspace,
                                size_t ws_bytes, void* cuda_stream, pflbm_batch** out) {
  if (!out || n <= 0 || !doms || !dev_workspace || ((uintptr_t)dev_workspace % kAlign) != 0)
    return PFLBM_EINVAL;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!doms[i] || doms[i]->storage != kFP32 || doms[i]->wall_x) {
      set_msg("pflbm_batch_create: every domain must exist, use FP32 storage and be "
              "periodic in x");
      return PFLBM_EINVAL;
    }
    if (!doms[i]->has_state) {
      set_msg("pflbm_batch_create: a domain has no initial state");
      return PFLBM_ESTATE;
    }
  }
  const size_t need = pflbm_batch_workspace_bytes(n, doms);
  if (ws_bytes < need) {
    set_msg("pflbm_batch_create: workspace too small");
    return PFLBM_ENOMEM_WS;
  }
  pflbm_batch* b = new (std::nothrow) pflbm_batch;
  if (!b) return PFLBM_EINVAL;
  memset(b, 0, sizeof(*b));
  b->n = n;
  b->doms = new (std::nothrow) pflbm_domain*[n];
  b->host_table = new (std::nothrow) StepArgs[2 * n];
  if (!b->doms || !b->host_table) {
    pflbm_batch_destroy(b);
    return PFLBM_EINVAL;
  }
  for (int i = 0; i < n; ++i) b->doms[i] = doms[i];
  b->stream = (cudaStream_t)cuda_stream;
  b->ws = (char*)dev_workspace;
  b->table_off = 0;
  b->mode = kGather;
  b->ctas_per_sm = batch_blocks_per_sm(kGather);
  b->rows = kTY;
  // one work-list per tile height, each sorted by force form, then by domain
  // and tile (row-major)
  size_t off = align_up(sizeof(StepArgs) * 2 * (size_t)n);
  for (int r = 0; r < 2; ++r) {
    const int rows = kBatchRows[r];
    long long items = 0;
    for (int i = 0; i < n; ++i) items += tiles_of(doms[i], rows);
    int4* h = new (std::nothrow) int4[items];
    if (!h) {
      pflbm_batch_destroy(b);
      return PFLBM_EINVAL;
    }
    long long k = 0;
    for (int form = 0; form < 8; ++form)
      for (int i = 0; i < n; ++i) {
        if (doms[i]->par.force != form) continue;
        const int ntx = (doms[i]->nx + kTX - 1) / kTX, nty = (doms[i]->ny + rows - 1) / rows;
        for (int ty = 0; ty < nty; ++ty)
          for (int tx = 0; tx < ntx; ++tx) h[k++] = make_int4(i, tx * kTX, ty * rows, form);
      }
    b->items_off[r] = off;
    b->nitems[r] = (int)k;
    off += align_up(sizeof(int4) * (size_t)k);
    b->tickets_off = off;
    cudaError_t e = cudaMemcpyAsync(b->ws + b->items_off[r], h, sizeof(int4) * k,
                                    cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    delete[] h;
    if (e != cudaSuccess) {
      set_err("pflbm_batch_create", e);
      pflbm_batch_destroy(b);
      return PFLBM_ECUDA;
    }
  }
  *out = b;
  return PFLBM_OK;
}

pflbm_status pflbm_batch_set_graphs(pflbm_batch* b, int enable) {
  if (!b) return PFLBM_EINVAL;
  if (enable && b->stream == nullptr) {
    set_msg("pflbm_batch_set_graphs: graphs need a non-default stream");
    return PFLBM_EINVAL;
  }
  b->graphs = enable != 0;
  batch_drop_graph(b);
  return PFLBM_OK;
}

pflbm_status pflbm_batch_set_config(pflbm_batch* b, int mode, int ctas_per_sm) {
  if (!b || mode < 0 || mode >= kNumBatchModes || ctas_per_sm < 1 ||
      ctas_per_sm > batch_blocks_per_sm(mode))
    return PFLBM_EINVAL;
  if (mode == kBoxes && b->rows != kTY) {
    set_msg("pflbm_batch_set_config: box staging needs tiles of the full height");
    return PFLBM_EINVAL;
  }
  b->mode = mode;
  b->ctas_per_sm = ctas_per_sm;
  batch_drop_graph(b);
  return PFLBM_OK;
}

pflbm_status pflbm_batch_set_tile_rows(pflbm_batch* b, int rows) {
  if (!b || (rows != kTY && rows != kShortRows)) return PFLBM_EINVAL;
  if (rows != kTY && b->mode == kBoxes) {
    set_msg("pflbm_batch_set_tile_rows: box staging needs tiles of the full height");
    return PFLBM_EINVAL;
  }
  b->rows = rows;
  batch_drop_graph(b);
  return PFLBM_OK;
}

int pflbm_batch_get_tile_rows(const pflbm_batch* b) { return b ? b->rows : -1; }

long long pflbm_batch_items(const pflbm_batch* b) {
  return b ? b->nitems[rows_slot(b->rows)] : -1;
}

pflbm_status pflbm_batch_step(pflbm_batch* b, int nsteps) {
  if (!b || nsteps < 0) return PFLBM_EINVAL;
  if (nsteps == 0) return PFLBM_OK;
  // the batch stream must see every domain's pending work
  bool any_first = false;
  for (int i = 0; i < b->n; ++i) {
    pflbm_domain* d = b->doms[i];
    any_first = any_first || d->t == 0;
    if (d->stream != b->stream) {
      cudaError_t e = cudaStreamSynchronize(d->stream);
      if (e != cudaSuccess) {
        set_err("pflbm_batch_step", e);
        return PFLBM_ECUDA;
      }
    }
  }
  cudaError_t e = cudaSuccess;
  int left = nsteps, bp = 0;
  if (any_first) {
    // first batch step with the first-step flag of the domains at t = 0
    e = upload_table(b, 0, 1);
    if (e == cudaSuccess) e = batch_launch(b, 0);
    bp = 1;
    --left;
  }
  if (e == cudaSuccess) e = upload_table(b, 0, 0);
  if (e == cudaSuccess && b->graphs && left >= kBatchGraphSteps + bp) {
    if (bp == 1) {  // graphs start from step parity 0
      e = batch_launch(b, 1);
      bp = 0;
      --left;
    }
    if (!b->gexec) {
      cudaGraph_t g = nullptr;
      e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
      for (int k = 0; k < kBatchGraphSteps && e == cudaSuccess; ++k) e = batch_launch(b, k & 1);
      cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
      if (e == cudaSuccess) e = e2;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) b->gexec = nullptr;
    }
    while (e == cudaSuccess && left >= kBatchGraphSteps) {
      e = cudaGraphLaunch(b->gexec, b->stream);
      left -= kBatchGraphSteps;  // even: step parity unchanged
    }
  }
  while (e == cudaSuccess && left > 0) {
    e = batch_launch(b, bp);
    bp ^= 1;
    --left;
  }
  if (e != cudaSuccess) {
    set_err("pflbm_batch_step", e);
    return PFLBM_ECUDA;
  }
  for (int i = 0; i < b->n; ++i) {
    b->doms[i]->cur ^= (nsteps & 1);
    b->doms[i]->t += nsteps;
    drop_graph(b->doms[i]);
  }
  return PFLBM_OK;
}

pflbm_status pflbm_batch_autotune(pflbm_batch* b, int trial_steps, int* mode_out,
                                  int* ctas_per_sm_out) {
  if (!b || trial_steps < 1) return PFLBM_EINVAL;
  for (int i = 0; i < b->n; ++i)
    if (b->doms[i]->t == 0) {
      set_msg("pflbm_batch_autotune: step the batch once before tuning");
      return PFLBM_ESTATE;
    }
  // trial steps write only the spare buffers and keep (phi u): state unchanged
  cudaError_t e = upload_table(b, 1, 0);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int keep_mode = b->mode, keep_cps = b->ctas_per_sm, keep_rows = b->rows;
  float best = 1e30f;
  int best_mode = keep_mode, best_cps = keep_cps, best_rows = keep_rows;
  // candidates: staging mode x tile rows (short tiles with gathers only) x
  // persistent CTAs per SM
  for (int m = 0; m < kNumBatchModes && e == cudaSuccess; ++m) {
    for (int r = 0; r < 2 && e == cudaSuccess; ++r) {
      if (m == kBoxes && kBatchRows[r] != kTY) continue;
      for (int cps = 1; cps <= batch_blocks_per_sm(m) && e == cudaSuccess; ++cps) {
        b->mode = m;
        b->rows = kBatchRows[r];
        b->ctas_per_sm = cps;
        e = batch_launch(b, 0);  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
        for (int k = 0; k < trial_steps && e == cudaSuccess; ++k) e = batch_launch(b, 0);
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best) {
          best = ms;
          best_mode = m;
          best_cps = cps;
          best_rows = kBatchRows[r];
        }
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  b->mode = e == cudaSuccess ? best_mode : keep_mode;
  b->ctas_per_sm = e == cudaSuccess ? best_cps : keep_cps;
  b->rows = e == cudaSuccess ? best_rows : keep_rows;
  batch_drop_graph(b);
  if (e != cudaSuccess) {
    set_err("pflbm_batch_autotune", e);
    return PFLBM_ECUDA;
  }
  if (mode_out) *mode_out = best_mode;
  if (ctas_per_sm_out) *ctas_per_sm_out = best_cps;
  return PFLBM_OK;
}

void pflbm_batch_destroy(pflbm_batch* b) {
  if (!b) return;
  batch_drop_graph(b);
  delete[] b->doms;
  delete[] b->host_table;
  delete b;
}

const char* pflbm_status_str(pflbm_status s) {
  switch (s) {
    case PFLBM_OK: return "ok";
    case PFLBM_EINVAL: return "invalid argument";
    case PFLBM_ENOMEM_WS: return "workspace too small";
    case PFLBM_ECUDA: return "CUDA error";
    case PFLBM_EUNSTABLE: return "non-finite state";
    case PFLBM_ETIMEOUT: return "device wait timed out";
    case PFLBM_ESTATE: return "call out of order";
  }
  return "unknown status";
}

const char* pflbm_last_error(void) { return g_err; }

const char* pflbm_version(void) { return "pflbm 0.1 sm_103a"; }

}  // extern "C"

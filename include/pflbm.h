/*
 * pflbm.h — C ABI of the GB300 (sm_103a) phase-field lattice Boltzmann step.
 *
 * The library advances the coupled D2Q9 populations of the phase-field
 * lattice Boltzmann method of Zhang, Liang & Guo (arXiv 2012.14729, Sec. 3):
 * the pressure-based flow populations f_i (He et al.) and the order-parameter
 * populations h_i (improved Cahn-Hilliard scheme), with the interfacial force
 * in any of the paper's eight formulations (Sec. 2.2) and half-way
 * bounce-back walls (Sec. 4).  One call of pflbm_step runs the fused CUDA
 * kernel once per time step on the caller's stream.
 *
 * Conventions shared by every entry point
 *   - Units: lattice units, delta x = delta t = 1, cs^2 = 1/3.
 *   - Layout of every field a caller passes or receives: float32, row-major
 *     [ny][nx], x fastest; population blocks are [9][ny][nx] in the D2Q9 order
 *     c_0..c_8 = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),(-1,-1),(1,-1).
 *   - Phases: phi = +1 in fluid 1, phi = -1 in fluid 2 (Sec. 2.1).
 *   - Ownership: the caller owns the device workspace (its size from
 *     pflbm_workspace_bytes), the CUDA stream and every input/output buffer.
 *     The library allocates no device memory and keeps no caller pointer
 *     beyond a call, except the workspace and stream given to pflbm_create,
 *     which must outlive the handle.  The handle itself is host memory
 *     released by pflbm_destroy.
 *   - Pointers flagged `on_device` are device pointers when the flag is
 *     nonzero and host pointers otherwise.
 *   - Asynchrony: pflbm_step only enqueues work on the stream.  Calls that
 *     return data to a host buffer (read, diagnostics, save_state to host)
 *     synchronise the stream before returning.
 *   - Errors: every call returns a pflbm_status; PFLBM_ECUDA carries the CUDA
 *     error text in pflbm_last_error().  Nothing aborts the process.
 *   - Threads: one handle must not be used from two host threads at once;
 *     distinct handles are independent.
 */
#ifndef PFLBM_H
#define PFLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pflbm_domain pflbm_domain;

typedef enum {
  PFLBM_OK = 0,
  PFLBM_EINVAL = 1,     /* bad argument or parameter */
  PFLBM_ENOMEM_WS = 2,  /* workspace smaller than pflbm_workspace_bytes */
  PFLBM_ECUDA = 3,      /* a CUDA call failed, see pflbm_last_error() */
  PFLBM_EUNSTABLE = 4,  /* a diagnostic found NaN or Inf in the state */
  PFLBM_ETIMEOUT = 5,   /* a bounded device wait expired */
  PFLBM_ESTATE = 6      /* call out of order (no params / no initial phi) */
} pflbm_status;

/* Boundaries: PERIODIC; WALL (y only): half-way bounce-back no-slip walls,
 * moving along x at uw_bottom / uw_top (Sec. 4); FREESLIP (x only):
 * free-slip side walls at x = -1/2 and nx - 1/2, planes of mirror symmetry
 * (specular reflection of the populations, mirror ghosts for the stencils),
 * as in the rising-bubble benchmark (Sec. 5.4).  Free-slip side walls need
 * gx = 0 and y-walls at rest, run the gather staging only, and are not
 * supported by batches or the adjoint. */
typedef enum { PFLBM_PERIODIC = 0, PFLBM_WALL = 1, PFLBM_FREESLIP = 2 } pflbm_bc;

/* Interfacial force formulations (Sec. 2.2):
 *   STF1  -div(kappa grad phi (x) grad phi)                    Eq. SF1
 *   STF2  div(kappa(|grad phi|^2 I - grad phi (x) grad phi))   Eq. SF2
 *   CPF1  -phi grad mu,   CPF2  mu grad phi                    Eq. SF3456
 *   PF1   -kappa grad phi lap phi, PF2 kappa phi grad lap phi  Eq. SF3456
 *   CSF1  -kappa grad phi |grad phi| div n                     Eq. SF7
 *   CSF2  -(sigma/2) grad phi div n                            Eq. SF8
 * A family name alone means its first variant. */
typedef enum {
  PFLBM_STF1 = 0, PFLBM_STF2 = 1, PFLBM_CPF1 = 2, PFLBM_CPF2 = 3,
  PFLBM_PF1 = 4, PFLBM_PF2 = 5, PFLBM_CSF1 = 6, PFLBM_CSF2 = 7,
  PFLBM_STF = PFLBM_STF1, PFLBM_CPF = PFLBM_CPF1, PFLBM_PF = PFLBM_PF1,
  PFLBM_CSF = PFLBM_CSF1
} pflbm_force;

/* How populations are stored in HBM.  Arithmetic is float32 in every case.
 * FP16/BF16 store f_i and h_1..h_8 as 16-bit scaled deviations from the rest
 * state (f^rest = 0, h_i^rest = 0 for i > 0), i.e. p_i / w_i * scale, and keep
 * h_0 (which carries phi) in float32. */
typedef enum { PFLBM_FP32 = 0, PFLBM_FP16 = 1, PFLBM_BF16 = 2 } pflbm_storage;

/* Fields of pflbm_read, all at the current time level (Eq. mac):
 * phi, rho, u_x, u_y, generalised pressure P_sf, chemical potential mu,
 * hydrodynamic pressure p_h (P_sf minus the gradient terms of the chosen
 * form, Eqs. SF1, SF2, P3456), interfacial + gravity force F_x, F_y. */
typedef enum {
  PFLBM_PHI = 0, PFLBM_RHO = 1, PFLBM_UX = 2, PFLBM_UY = 3, PFLBM_P = 4,
  PFLBM_MU = 5, PFLBM_PH = 6, PFLBM_FX = 7, PFLBM_FY = 8, PFLBM_NFIELDS = 9
} pflbm_field;

/* Physical parameters in lattice units (Sec. 2.1, Sec. 3):
 *   sigma, W       surface tension and interface width; beta = 3 sigma/(4W),
 *                  kappa = 3 W sigma / 8
 *   M, tau_h       mobility and CH relaxation time; eta = M / (cs^2 (tau_h - 1/2))
 *   rho1, rho2     densities of fluid 1 (phi = +1) and fluid 2 (phi = -1)
 *   nu1, nu2       kinematic viscosities; tau_f = 1/2 + mu(phi) / (rho cs^2)
 *   gx, gy         gravity, F_g = (rho - rho0) g
 *   rho0           background density; NaN selects the domain mean of rho(phi0)
 *   uw_bottom/top  x-velocity of the walls at y = -1/2 and y = ny - 1/2
 *   eps            regularisation of the CSF normal n = grad phi / sqrt(|grad phi|^2 + eps^2)
 *   force          a pflbm_force
 *   scale_f, scale_h  16-bit storage scales (powers of two); 0 selects 2^round(log2(4/sigma)) */
typedef struct {
  double sigma, W, M, tau_h;
  double rho1, rho2, nu1, nu2;
  double gx, gy, rho0;
  double uw_bottom, uw_top;
  double eps;
  int32_t force;
  int32_t reserved;
  double scale_f, scale_h;
} pflbm_params;

/* Geometry of the Laplace-law measurement (Sec. 5.1): the pressure jump is
 * the mean p_h over nodes within r_in of (xc, yc) minus the mean over nodes
 * farther than r_out (periodic distances). */
typedef struct {
  double xc, yc, r_in, r_out;
} pflbm_diag_geom;

/* FP64 diagnostics of the current state (Secs. 5.1, 5.2, 5.5). */
typedef struct {
  double mass;        /* sum phi (conserved exactly in exact arithmetic) */
  double umax;        /* max |u| (spurious currents) */
  double area1;       /* sum (1 + phi)/2: area of fluid 1 */
  double R_num;       /* sqrt(area1 / pi) */
  double p_in, p_out; /* mean p_h inside r_in / outside r_out */
  double dp;          /* p_in - p_out */
  double sigma_num;   /* R_num * dp (Laplace law) */
  double xc1, yc1;    /* centroid of fluid 1 (weight (1 + phi)/2) */
  double taylor_D;    /* (L - B)/(L + B), L, B = 4 sqrt(eigenvalues of the
                         second-moment matrix of (1 + phi)/2) */
  double nonfinite;   /* number of nodes with a NaN/Inf field */
} pflbm_diag;

/* Rising-bubble benchmark quantities (Sec. 5.4), lattice units (node
 * spacing 1, node (x, y) at coordinates x, y).  Fluid 2 (phi = -1) is the
 * bubble.  The phi = 0 contour is traced by marching squares over the cells
 * of the node lattice (one cell per node, the node its lower-left corner;
 * cells wrap in a periodic direction, none lie beyond the last node towards
 * a wall): a corner is inside when phi < 0, the contour crosses each edge
 * whose ends differ at the zero of the linear interpolant, and a cell with
 * four crossings is paired by the sign of its corner mean (inside: the
 * segments cut off the outside corners). */
typedef struct {
  double mass2;       /* sum (1 - phi) */
  double xc2, yc2;    /* centre of mass: sum (1 - phi) x / mass2, likewise y
                         (Eq. quantify-yc); 0 when mass2 = 0 */
  double uc2, vc2;    /* sum (1 - phi) u_x / mass2, likewise u_y: the rise
                         velocity v_c (Eq. quantify-uc) */
  double area2;       /* number of nodes with phi < 0 */
  double perimeter;   /* length of the phi = 0 contour */
  double circularity; /* 2 sqrt(pi area2) / perimeter (Eq. circularity);
                         0 without a contour */
  double nonfinite;   /* nodes with a NaN/Inf phi or u (their cells add nothing) */
} pflbm_bubble_diag;

/* ---- domain ------------------------------------------------------------ */

/* Bytes of device workspace a domain of nx x ny with this storage needs
 * (populations double-buffered with one ghost row above and below, phi u,
 * field staging and reduction scratch).  0 for invalid sizes: nx, ny >= 4
 * and 9 (ny + 2) nx < 2^31 (population planes use 32-bit offsets; about
 * 238 M nodes). */
size_t pflbm_workspace_bytes(int nx, int ny, pflbm_storage storage);

/* Create a domain over a caller-owned device workspace (256-byte aligned,
 * at least pflbm_workspace_bytes) and CUDA stream (cudaStream_t, NULL = the
 * legacy default stream).  bc_x is PFLBM_PERIODIC or PFLBM_FREESLIP; bc_y is
 * PFLBM_PERIODIC or PFLBM_WALL.
 * nx, ny >= 4.  The domain (Sec. 5 benchmarks) is the paper's uniform
 * L_x x L_y lattice.  Errors: EINVAL, ENOMEM_WS. */
pflbm_status pflbm_create(int nx, int ny, pflbm_bc bc_x, pflbm_bc bc_y,
                          pflbm_storage storage, void* dev_workspace,
                          size_t ws_bytes, void* cuda_stream, pflbm_domain** out);

/* Set the physical parameters (copied).  Rejects sigma < 0, W <= 0, M <= 0,
 * tau_h <= 1/2, non-positive densities or viscosities, eps < 0, an unknown
 * force, and non-power-of-two storage scales, with EINVAL. */
pflbm_status pflbm_set_params(pflbm_domain* d, const pflbm_params* p);

/* Initial state (Sec. 5.1: zero velocity): f = f^eq(P = 0, u = 0) = 0 and
 * h = h^eq(phi0, mu0, u = 0), mu0 the chemical potential of phi0
 * (Eq. chemical_potential).  phi0: [ny][nx] float32.  Resets the step count.
 * Errors: ESTATE without params, ECUDA. */
pflbm_status pflbm_init_phi(pflbm_domain* d, const float* phi0, int on_device);

/* Advance nsteps time steps (Eqs. fh; one fused kernel per step), enqueued
 * on the stream.  With graphs enabled the steps after the first replay a
 * captured CUDA graph.  Errors: ESTATE before init, ECUDA. */
pflbm_status pflbm_step(pflbm_domain* d, int nsteps);

/* Use captured CUDA graphs for pflbm_step (1) or plain launches (0, the
 * default).  Graphs need a non-default stream. */
pflbm_status pflbm_set_graphs(pflbm_domain* d, int enable);

/* How the fused step kernel obtains the populations it pulls:
 *   PFLBM_STAGE_BOXES   TMA box loads of each tile's population planes into
 *                       shared memory, persistent CTAs (2 per SM)
 *   PFLBM_STAGE_GATHER  L1-cached gathers straight from the planes, one CTA
 *                       of 256 threads per tile, two collision nodes per
 *                       thread (the default)
 *   PFLBM_STAGE_GATHER8 the same gathers on 32 x 8 tiles, one CTA of 256
 *                       threads per tile and one collision node per thread:
 *                       each thread pulls its own node first and keeps its
 *                       populations in registers for the collision, which
 *                       then re-reads no plane (finer-grained waves on
 *                       lattices of a few hundred tiles)
 *   PFLBM_STAGE_MARCH   persistent CTAs sweep column strips along y; the
 *                       pulled population rows are copied two iterations
 *                       ahead into a ring in shared memory (cp.async), the
 *                       y halo of phi and its derived fields is kept in row
 *                       rings.
 *                       Needs periodic x with nx a multiple of 4 (float32)
 *                       or 8 (16-bit storage), ny >= 8, no side walls;
 *                       EINVAL otherwise.  The batch refuses it.
 * All compute the same step; results agree to float32 rounding order. */
enum {
  PFLBM_STAGE_BOXES = 0,
  PFLBM_STAGE_GATHER = 1,
  PFLBM_STAGE_MARCH = 2,
  PFLBM_STAGE_GATHER8 = 3
};
pflbm_status pflbm_set_stage_mode(pflbm_domain* d, int mode);
int pflbm_get_stage_mode(const pflbm_domain* d);

/* Time trial_steps steps of every stage mode on this domain's current state
 * and keep the fastest (written to *mode_out if not NULL).  Trial steps write
 * only the spare population buffer, so the state and step count are
 * unchanged.  Synchronises the stream.  Errors: ESTATE before init, ECUDA. */
pflbm_status pflbm_autotune(pflbm_domain* d, int trial_steps, int* mode_out);

/* In PFLBM_STAGE_BOXES, stage interior tiles with TMA tensor loads (1, the
 * default where the row pitch nx * element size is a multiple of 16 bytes)
 * or fill every tile with cp.async / plain loads (0).  Both fill identical
 * shared-memory boxes, so results are bitwise equal; the switch exists to
 * test exactly that. */
pflbm_status pflbm_set_tma(pflbm_domain* d, int enable);

/* Steps taken since pflbm_init_phi. */
long long pflbm_steps_done(const pflbm_domain* d);

/* One field at the current time level into dst [ny][nx] (synchronises when
 * dst is on the host).  Errors: EINVAL for an unknown field, ESTATE, ECUDA. */
pflbm_status pflbm_read(pflbm_domain* d, pflbm_field field, float* dst, int on_device);

/* All PFLBM_NFIELDS fields into dst [PFLBM_NFIELDS][ny][nx]. */
pflbm_status pflbm_read_fields(pflbm_domain* d, float* dst, int on_device);

/* The pre-collision populations at the current time level, decoded to
 * float32: f_out and h_out [9][ny][nx] (either may be NULL). */
pflbm_status pflbm_read_populations(pflbm_domain* d, float* f_out, float* h_out,
                                    int on_device);

/* FP64 diagnostics of the current state; geom may be NULL (no pressure
 * jump).  Synchronises.  Returns EUNSTABLE if any node is non-finite (the
 * struct is still filled). */
pflbm_status pflbm_diagnostics(pflbm_domain* d, const pflbm_diag_geom* geom,
                               pflbm_diag* out);

/* Rising-bubble quantities of the current state (FP64 sums of the float32
 * fields, deterministic order).  Synchronises.  Uses the same workspace
 * scratch as pflbm_diagnostics.  Returns EUNSTABLE if any node is
 * non-finite (the struct is still filled); ESTATE before init. */
pflbm_status pflbm_bubble_diagnostics(pflbm_domain* d, pflbm_bubble_diag* out);

/* Checkpoint / resume: the raw state (populations in their storage format,
 * phi u, step count, and the mean of phi0 from which the default rho0
 * follows).  pflbm_state_bytes gives the size of the blob.  Loading needs
 * the parameters set first; when they leave rho0 to the library (NaN), the
 * resumed run takes rho0 = rho(mean phi0) of the run that saved the blob,
 * with the current rho1, rho2.  Errors: EINVAL for a blob of another size,
 * storage or boundary kind, ESTATE without parameters, ECUDA. */
size_t pflbm_state_bytes(const pflbm_domain* d);
pflbm_status pflbm_save_state(pflbm_domain* d, void* dst, int on_device);
pflbm_status pflbm_load_state(pflbm_domain* d, const void* src, int on_device);

void pflbm_destroy(pflbm_domain* d);

/* ---- adjoint: gradients of objectives of the final phi ------------------- */

/* Device scratch of pflbm_adjoint_run: a checkpoint at the start of every
 * segment of ckpt_every steps but the last, the tape of one segment (24
 * float32 planes of nx * ny per step: pulled f, phi, grad phi, lap phi, mu,
 * force values, u, P, div(phi u), d_t(phi u)), a second such tape when there
 * are two segments or more, two adjoint states and work planes.  0 for invalid input: FP32 storage, periodic x, nsteps and
 * ckpt_every >= 1, and 24 nx ny < 2^31 (the tape's 32-bit plane offsets;
 * about 89 M nodes). */
size_t pflbm_adjoint_scratch_bytes(const pflbm_domain* d, int nsteps, int ckpt_every);

/* Run nsteps steps from phi0 (device [ny][nx]) with the domain's parameters,
 * checkpointing every ckpt_every steps, then run the hand-written discrete
 * adjoint of the step (Sec. 3 scheme, every force form, periodic or walls)
 * backwards through the steps.  Each segment but the last is recomputed from
 * its checkpoint by a taping step that records the step's intermediates; the
 * last is taped during the forward run (ckpt_every >= nsteps: no
 * recomputation at all).  The recomputation of a segment runs on a stream the
 * call creates (and destroys before returning) while the domain's stream
 * reverses the segment after it, into the other of the two tapes.
 * Recomputation and reverse sweep of a segment are replayed from CUDA graphs
 * where the stream can be captured (the reverse sweep not on the legacy
 * default stream); the first use in a call captures them.
 * Input dJ_dphiT: gradient of an objective J with respect to the final phi_T
 * (device [ny][nx]).  Outputs: dJ_dphi0 (device [ny][nx]) and, on the host,
 * dJ/dsigma and dJ/dM (FP64 accumulation; sigma through beta, kappa and the
 * CSF-2 prefactor; M through eta).  rho0 and g are held fixed.  On return the
 * domain holds the final state of the forward run.  Synchronises.  Errors:
 * EINVAL, ESTATE (no parameters), ENOMEM_WS (scratch), ECUDA. */
pflbm_status pflbm_adjoint_run(pflbm_domain* d, const float* phi0, int nsteps, int ckpt_every,
                               const float* dJ_dphiT, float* dJ_dphi0, double* dJ_dsigma,
                               double* dJ_dM, void* scratch, size_t scratch_bytes);

/* ---- batch: many independent domains, one launch per time step ---------- */

typedef struct pflbm_batch pflbm_batch;

/* Device scratch a batch of these n domains needs: two argument records per
 * domain, one work item per (domain, tile) and the kernel's item counter. */
size_t pflbm_batch_workspace_bytes(int n, pflbm_domain* const* doms);

/* Group n domains (FP32 storage, parameters and initial state set; sizes and
 * force forms may all differ) into a batch whose steps run on cuda_stream.
 * Each step is ONE persistent launch: CTAs claim (domain, tile) items of a
 * work-list sorted by force form from a counter in the workspace, which the
 * step zeroes on cuda_stream before the launch.  The domains keep their own state and
 * remain usable one by one (diagnostics, read-back) once the batch stream
 * has been synchronised; stepping a domain alone between batch steps is
 * allowed.  The batch keeps the domain handles and the workspace until
 * pflbm_batch_destroy.  Errors: EINVAL (bad domain list, 16-bit storage),
 * ESTATE (a domain without state), ENOMEM_WS. */
pflbm_status pflbm_batch_create(int n, pflbm_domain* const* doms, void* dev_workspace,
                                size_t ws_bytes, void* cuda_stream, pflbm_batch** out);

/* Advance every domain of the batch by nsteps steps (domains still at step 0
 * first take one step of their own, which fixes d_t(phi u) = 0 there). */
pflbm_status pflbm_batch_step(pflbm_batch* b, int nsteps);

/* Replay captured CUDA graphs of batch steps (1) or launch each step (0). */
pflbm_status pflbm_batch_set_graphs(pflbm_batch* b, int enable);

/* Staging mode (PFLBM_STAGE_*) and persistent CTAs per SM of the batch
 * kernel (EINVAL for box staging while the tiles are short). */
pflbm_status pflbm_batch_set_config(pflbm_batch* b, int mode, int ctas_per_sm);

/* Tile shape of the batch: 32 x 16 tiles (rows = 16, the default; two
 * collision nodes per thread) or 32 x 8 tiles (rows = 8; one node per
 * thread, gather staging only, EINVAL with box staging).  Both compute the
 * same step. */
pflbm_status pflbm_batch_set_tile_rows(pflbm_batch* b, int rows);
int pflbm_batch_get_tile_rows(const pflbm_batch* b);

/* Time trial steps of every candidate (staging mode x tile rows x CTAs per
 * SM) on the current states, which stay unchanged, and keep the fastest;
 * the outputs (each may be NULL) receive the mode and CTAs per SM, and
 * pflbm_batch_get_tile_rows the tile rows.  ESTATE before the first batch
 * step. */
pflbm_status pflbm_batch_autotune(pflbm_batch* b, int trial_steps, int* mode_out,
                                  int* ctas_per_sm_out);

/* Work items (domain tiles of the current shape) of one batch step. */
long long pflbm_batch_items(const pflbm_batch* b);

void pflbm_batch_destroy(pflbm_batch* b);

/* ---- diagnostics without allocation -------------------------------------- */

/* Largest lattice (nx * ny nodes) pflbm_field_diagnostics_noalloc accepts:
 * its reduction scratch is one fixed 4 MiB device array (one 128-byte row of
 * partial sums per 256 nodes), 4096 x 2048 nodes at most. */
#define PFLBM_NOALLOC_MAX_NODES 8388608

/* The FP64 diagnostics of pflbm_diagnostics (same sums, same pflbm_diag),
 * computed from fields the caller already holds on the device, without
 * allocating anything and without a domain or workspace.  The paper has no
 * counterpart: this is a library service, not part of the method.
 *
 * Who needs it: code that watches a running simulation from outside it, such
 * as a monitor thread or a host application that owns the whole device
 * memory budget.  There cudaMalloc can fail because the lattice holds nearly
 * all of HBM, and cudaFree waits for the whole device, so a per-call
 * allocation would stall the simulation's own streams.  Such callers cannot
 * lend this call a workspace either; it uses a 4 MiB device array compiled
 * into the library instead, and a call makes no cudaMalloc, cudaFree or other
 * allocating call.
 *
 *   nx, ny  lattice size; nx * ny <= PFLBM_NOALLOC_MAX_NODES, else EINVAL
 *           with the limit in pflbm_last_error()
 *   bc_x    PFLBM_PERIODIC or PFLBM_FREESLIP, bc_y PFLBM_PERIODIC or
 *           PFLBM_WALL: the sides of the lattice the fields come from; the
 *           distance to the pressure-jump centre wraps only across periodic
 *           sides (as in pflbm_diagnostics)
 *   fields  device memory of the current device, [PFLBM_NFIELDS][ny][nx]
 *           float32 as pflbm_read_fields writes it (slots phi, ux, uy, P,
 *           p_h are read); borrowed; a host pointer is rejected with EINVAL
 *   geom    pressure-jump geometry or NULL; out: host struct, filled
 *   stream  cudaStream_t to run on (NULL: the legacy default stream); the
 *           call synchronises it before returning
 *
 * Set-up: every call looks up the array's address on the current device
 * (cudaGetSymbolAddress).  The first call on a device loads the library's
 * module that holds the array, and with CUDA's lazy module loading that is
 * when the driver reserves the array's 4 MiB on the device; later calls only
 * find it.  Make that first call before the simulation fills HBM and before
 * any stream capture.  A device reset (cudaDeviceReset, or a reset of the
 * primary context) unloads the module: the next call loads it again and is a
 * first call in this sense.  The array is shared by every caller in the
 * process on that device and keeps the last call's partial sums (a call
 * clears the counter it needs itself): calls that overlap (from two host
 * threads, or on two streams without ordering between them) race on it and
 * may return wrong values; serialise them.  Returns EUNSTABLE if a node is
 * non-finite (the struct is still filled), ECUDA on a CUDA error. */
pflbm_status pflbm_field_diagnostics_noalloc(int nx, int ny, pflbm_bc bc_x, pflbm_bc bc_y,
                                             const float* fields, const pflbm_diag_geom* geom,
                                             pflbm_diag* out, void* stream);

/* ---- misc ---------------------------------------------------------------- */

const char* pflbm_status_str(pflbm_status s);
const char* pflbm_last_error(void);
/* Library version and the device architecture it was compiled for. */
const char* pflbm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PFLBM_H */

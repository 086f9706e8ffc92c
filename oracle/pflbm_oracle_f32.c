/*
 * Float32-state build of the oracle, for deriving parity tolerances.
 *
 * TEST INFRASTRUCTURE ONLY (same rules as pflbm_oracle.c).  This file
 * compiles the unchanged oracle source with every `double` declaration read
 * as `float`, so that populations, fields and (phi u) are stored in float32
 * while the algorithm, its order of passes and its operations stay those of
 * the FP64 oracle.  Comparing such a run with the FP64 oracle measures how far
 * float32 rounding alone moves a workload; tests use it to set the tolerance
 * of the float32 CUDA path on workloads where that deviation exceeds the
 * fixed bar.  The exported w32_* functions keep double arrays at the interface.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* the system headers are already included, so the oracle's own #includes are
 * no-ops and only its declarations are re-typed */
#define double float
#include "pflbm_oracle.c"
#undef double

static float* to32(const double* a, size_t n) {
  float* b = (float*)malloc(n * sizeof(float));
  for (size_t i = 0; i < n; ++i) b[i] = (float)a[i];
  return b;
}
static void from32(double* a, const float* b, size_t n) {
  for (size_t i = 0; i < n; ++i) a[i] = b[i];
}

void w32_step(const double* p, int nx, int ny, int wall, double* f, double* h, double* pu,
              int nsteps, int first) {
  size_t n = (size_t)nx * ny;
  float *pf = to32(p, P_NPAR), *ff = to32(f, 9 * n), *hh = to32(h, 9 * n), *uu = to32(pu, 2 * n);
  orc_step(pf, nx, ny, wall, ff, hh, uu, nsteps, first);
  from32(f, ff, 9 * n);
  from32(h, hh, 9 * n);
  from32(pu, uu, 2 * n);
  free(pf);
  free(ff);
  free(hh);
  free(uu);
}

void w32_macro(const double* p, int nx, int ny, int wall, const double* f, const double* h,
               const double* pu, int first, double* out) {
  size_t n = (size_t)nx * ny;
  float *pf = to32(p, P_NPAR), *ff = to32(f, 9 * n), *hh = to32(h, 9 * n), *uu = to32(pu, 2 * n);
  float* o = (float*)malloc(sizeof(float) * M_NFIELDS * n);
  orc_macro(pf, nx, ny, wall, ff, hh, uu, first, o);
  from32(out, o, M_NFIELDS * n);
  free(pf);
  free(ff);
  free(hh);
  free(uu);
  free(o);
}

/* A plain C caller of the library: the boundary is a C ABI, usable without
 * Python.  One small reconstruction (N = 64, Np = 8) from host buffers:
 * plan, intensities, the default padded-box support, 20 iterations with their
 * error history, the 3D assembly into host memory, the state read back; and
 * the refusal of a NULL plan.  Prints "ok <first error> <last error>" and
 * returns 0, or prints the library's message and returns 1. */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include "cpra.h"

#define N 64
#define NP 8
#define ITERS 20

static int check(cpra_status st, cpra_plan_t plan, const char* what) {
  if (st == CPRA_OK) return 0;
  fprintf(stderr, "%s: status %d: %s\n", what, (int)st, cpra_last_error(plan));
  return 1;
}

int main(void) {
  float* I = malloc(sizeof(float) * NP * N * N);
  double* err = malloc(sizeof(double) * ITERS * NP);
  float* g = malloc(sizeof(float) * NP * N * N);
  float* vol = malloc(sizeof(float) * 2 * N * N * N);
  if (!I || !err || !g || !vol) return 1;
  /* centred patterns: a Gaussian bump whose width varies with the angle */
  for (int n = 0; n < NP; ++n)
    for (int y = 0; y < N; ++y)
      for (int x = 0; x < N; ++x) {
        const double r2 = (double)(x - N / 2) * (x - N / 2) + (double)(y - N / 2) * (y - N / 2);
        I[((size_t)n * N + y) * N + x] = (float)(1e4 * exp(-r2 / (30.0 + 2.0 * n)) + 1.0);
      }
  if (cpra_iterate(NULL, 1, NULL) != CPRA_ERR_INVALID_ARG) {
    fprintf(stderr, "a NULL plan was not refused\n");
    return 1;
  }
  cpra_config cfg;
  cpra_plan_t plan = NULL;
  if (check(cpra_default_config(N, NP, &cfg), NULL, "default config")) return 1;
  cfg.hio_iters = 10;
  cfg.er_iters = 10;
  if (check(cpra_plan(&cfg, NULL, &plan), NULL, "plan")) return 1;
  int bad = check(cpra_load_intensities(plan, I, 0, NP, NULL), plan, "intensities");
  if (!bad) bad = check(cpra_load_support(plan, NULL, 0), plan, "support");
  if (!bad) bad = check(cpra_iterate(plan, ITERS, err), plan, "iterate");
  if (!bad) bad = check(cpra_assemble_3d(plan, vol), plan, "assemble");
  if (!bad) bad = check(cpra_result(plan, CPRA_RESULT_STATE, g, sizeof(float) * NP * N * N), plan, "result");
  if (!bad) {
    for (size_t i = 0; i < (size_t)ITERS * NP; ++i)
      if (!isfinite(err[i]) || err[i] < 0) bad = 1;
    for (size_t i = 0; i < (size_t)NP * N * N; ++i)
      if (!isfinite(g[i])) bad = 1;
    for (size_t i = 0; i < (size_t)2 * N * N * N; ++i)
      if (!isfinite(vol[i])) bad = 1;
    if (bad) fprintf(stderr, "non-finite output\n");
  }
  double e0 = 0.0, e1 = 0.0;
  for (int n = 0; n < NP; ++n) {
    e0 += err[n] / NP;
    e1 += err[(size_t)(ITERS - 1) * NP + n] / NP;
  }
  cpra_destroy(plan);
  free(I);
  free(err);
  free(g);
  free(vol);
  if (bad) return 1;
  printf("ok %.6e %.6e\n", e0, e1);
  return 0;
}

/* A plain C program on the library's C ABI (include/lcs.h), no Python:
 * particles released with the fluid velocity of a uniform flow keep it
 * (Eqs. 5-6 with U - V = 0 and no gravity), so after n steps of dt every
 * particle sits at X0 + n dt U0, unwrapped with its periodic image counts,
 * while it has migrated between the 2x2x2 subdomains and been cell-sorted.
 * Some particles are released in other periodic images of the box (the
 * library folds them in and counts the folds as images).  The final state is
 * read twice: in storage order (lcs_get_state, with image counts) and in
 * particle-id order, unwrapped (lcs_get_state_by_id).
 * Exit status 0 and "ok" on success. */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime_api.h>

#include "lcs.h"

#define CHECK(call)                                                          \
  do {                                                                       \
    int rc_ = (int)(call);                                                   \
    if (rc_ != 0) {                                                          \
      fprintf(stderr, "%s failed: %d\n", #call, rc_);                        \
      return 1;                                                              \
    }                                                                        \
  } while (0)

static double uniform01(uint64_t *s) { /* 64-bit LCG, top 53 bits */
  *s = *s * 6364136223846793005ULL + 1442695040888963407ULL;
  return (double)(*s >> 11) * (1.0 / 9007199254740992.0);
}

int main(void) {
  const int N = 16, steps = 50;
  const int64_t np = 4096;
  const double L = 2.0 * 3.14159265358979323846, dt = 0.01;
  const double U0[3] = {0.3, -0.2, 0.1};
  const size_t ncell = (size_t)N * N * N;
  double *field = malloc(3 * ncell * sizeof(double));
  double *x0 = malloc(3 * (size_t)np * sizeof(double));
  double *v0 = malloc(3 * (size_t)np * sizeof(double));
  uint64_t seed = 12345;
  for (int c = 0; c < 3; ++c) {
    for (size_t i = 0; i < ncell; ++i) field[c * ncell + i] = U0[c];
    for (int64_t p = 0; p < np; ++p) {
      /* images -2 .. 2 of the box by particle index */
      x0[c * np + p] = L * uniform01(&seed) + L * (double)((p + c) % 5 - 2);
      v0[c * np + p] = U0[c];
    }
  }
  double *d_field, *d_x0, *d_v0;
  CHECK(cudaMalloc((void **)&d_field, 3 * ncell * sizeof(double)));
  CHECK(cudaMalloc((void **)&d_x0, 3 * (size_t)np * sizeof(double)));
  CHECK(cudaMalloc((void **)&d_v0, 3 * (size_t)np * sizeof(double)));
  CHECK(cudaMemcpy(d_field, field, 3 * ncell * sizeof(double), cudaMemcpyHostToDevice));
  CHECK(cudaMemcpy(d_x0, x0, 3 * (size_t)np * sizeof(double), cudaMemcpyHostToDevice));
  CHECK(cudaMemcpy(d_v0, v0, 3 * (size_t)np * sizeof(double), cudaMemcpyHostToDevice));

  lcs_desc d;
  memset(&d, 0, sizeof d);
  d.n = N;
  d.box = L;
  d.sub[0] = d.sub[1] = d.sub[2] = 2;
  d.np = np;
  d.field_dtype = LCS_F64;
  d.field_kernel = LCS_KERNEL_AUTO;
  d.field = d_field;
  d.x0 = d_x0;
  d.v0 = d_v0;
  d.tau_const = 0.1;
  d.dt = dt;
  d.sort_every = 5;
  d.track_images = 1;
  lcs_ctx *ctx = NULL;
  CHECK(lcs_init(&d, 1, NULL, &ctx));
  CHECK(lcs_step(ctx, steps));
  CHECK(lcs_sync(ctx));

  double *x = malloc(3 * (size_t)np * sizeof(double));
  double *v = malloc(3 * (size_t)np * sizeof(double));
  uint32_t *ids = malloc((size_t)np * sizeof(uint32_t));
  int32_t *img = malloc(3 * (size_t)np * sizeof(int32_t));
  int64_t seg[9];
  CHECK(lcs_get_state(ctx, 0, x, v, NULL, ids, img, seg));

  int bad = 0;
  char *seen = calloc((size_t)np, 1);
  if (seg[0] != 0 || seg[8] != np) bad |= 1;
  for (int s = 0; s < 8; ++s)
    if (seg[s + 1] < seg[s]) bad |= 1;
  double ex = 0.0, ev = 0.0;
  for (int64_t i = 0; i < np; ++i) {
    const uint32_t id = ids[i];
    if (id >= (uint32_t)np || seen[id]) {
      bad |= 2;
      continue;
    }
    seen[id] = 1;
    for (int c = 0; c < 3; ++c) {
      const double want = x0[c * np + id] + steps * dt * U0[c];
      const double got = x[c * np + i] + L * img[c * np + i];
      ex = fmax(ex, fabs(got - want));
      ev = fmax(ev, fabs(v[c * np + i] - U0[c]));
    }
  }
  /* the same final state in particle-id order, unwrapped */
  double *xi = malloc(3 * (size_t)np * sizeof(double));
  double *vi = malloc(3 * (size_t)np * sizeof(double));
  uint32_t *idi = malloc((size_t)np * sizeof(uint32_t));
  CHECK(lcs_get_state_by_id(ctx, 0, xi, vi, idi));
  for (int64_t p = 0; p < np; ++p) {
    if (idi[p] != (uint32_t)p) bad |= 16;
    for (int c = 0; c < 3; ++c) {
      const double want = x0[c * np + p] + steps * dt * U0[c];
      ex = fmax(ex, fabs(xi[c * np + p] - want));
      ev = fmax(ev, fabs(vi[c * np + p] - U0[c]));
    }
  }
  if (!(ex < 1e-11)) bad |= 4;
  if (!(ev < 1e-13)) bad |= 8;
  lcs_destroy(ctx);
  free(xi);
  free(vi);
  free(idi);
  cudaFree(d_field);
  cudaFree(d_x0);
  cudaFree(d_v0);
  printf("%s: %lld particles, %d steps, max |dx| %.2e, max |dv| %.2e\n", bad ? "FAILED" : "ok",
         (long long)np, steps, ex, ev);
  return bad;
}

/*
 * A C caller of libamr that uses nothing but include/amr.h: a complete octree
 * of depth 3 with uniform density 1 (float64), an axis-aligned view of the
 * whole box at the deepest level, rendered into host buffers.  Closed form: a
 * ray crosses the unit box along +z, so every pixel's column is 1 and it
 * crosses 2^3 = 8 leaves; a batch of the same view in the three precisions
 * agrees.  Exit status 0 on success.
 */
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "amr.h"

enum { DEPTH = 3, N = 32 };

static int fail(const char* what, amr_status st) {
  fprintf(stderr, "%s failed: %d (%s)\n", what, (int)st, amr_last_error(NULL));
  return 1;
}

int main(void) {
  /* breadth-first complete tree: levels 1..DEPTH, 1 + 8 + 64 octs */
  int64_t n_oct = 0, per = 1;
  for (int l = 1; l <= DEPTH; ++l, per *= 8) n_oct += per;
  uint8_t* level = malloc((size_t)n_oct);
  int32_t* coord = malloc((size_t)n_oct * 3 * sizeof(int32_t));
  int32_t* child = malloc((size_t)n_oct * 8 * sizeof(int32_t));
  double* rho = malloc((size_t)n_oct * 8 * sizeof(double));
  if (!level || !coord || !child || !rho) return 1;
  level[0] = 1;
  coord[0] = coord[1] = coord[2] = 0;
  int64_t next = 1;
  for (int64_t o = 0; o < n_oct; ++o) {
    for (int c = 0; c < 8; ++c) {
      rho[o * 8 + c] = 1.0;
      child[o * 8 + c] = -1;
      if (level[o] < DEPTH) {
        child[o * 8 + c] = (int32_t)next;
        level[next] = (uint8_t)(level[o] + 1);
        for (int a = 0; a < 3; ++a) coord[next * 3 + a] = 2 * (coord[o * 3 + a] + ((c >> a) & 1));
        ++next;
      }
    }
  }
  amr_ctx* ctx = NULL;
  amr_status st = amr_create(&ctx, 0);
  if (st != AMR_OK) return fail("amr_create", st);
  const void* fields[1] = {rho};
  st = amr_load_octree(ctx, n_oct, level, coord, child, 1, fields, AMR_F64);
  if (st != AMR_OK) return fail("amr_load_octree", st);

  amr_camera cam;
  memset(&cam, 0, sizeof cam);
  cam.centre[0] = cam.centre[1] = cam.centre[2] = 0.5;
  cam.u[0] = 1.0;
  cam.v[1] = 1.0;
  cam.w[2] = 1.0;
  cam.fov[0] = cam.fov[1] = 1.0;
  cam.nx = cam.ny = N;
  cam.max_level = DEPTH;
  cam.mode = AMR_MODE_COLUMN;
  cam.precision = AMR_PREC_FP64;
  double map[N * N];
  int32_t counts[N * N];
  st = amr_render(ctx, &cam, map, counts, 0, NULL);
  if (st != AMR_OK) return fail("amr_render", st);
  for (int p = 0; p < N * N; ++p) {
    if (fabs(map[p] - 1.0) > 1e-12 || counts[p] != 8) {
      fprintf(stderr, "pixel %d: column %.17g, %d leaves\n", p, map[p], counts[p]);
      return 1;
    }
  }

  amr_camera cams[3] = {cam, cam, cam};
  cams[1].precision = AMR_PREC_FP32_KAHAN;
  cams[2].precision = AMR_PREC_FP32_PLAIN;
  double m0[N * N];
  float m1[N * N], m2[N * N];
  void* maps[3] = {m0, m1, m2};
  int32_t c0[N * N], c1[N * N], c2[N * N];
  int32_t* cnts[3] = {c0, c1, c2};
  st = amr_render_batch(ctx, 3, cams, maps, cnts, 0, NULL);
  if (st != AMR_OK) return fail("amr_render_batch", st);
  for (int p = 0; p < N * N; ++p) {
    if (c0[p] != 8 || c1[p] != 8 || c2[p] != 8 || fabs(m0[p] - 1.0) > 1e-12 || fabsf(m1[p] - 1.0f) > 1e-6f ||
        fabsf(m2[p] - 1.0f) > 1e-5f) {
      fprintf(stderr, "batch pixel %d differs\n", p);
      return 1;
    }
  }
  char stats[4096];
  st = amr_stats(ctx, stats, sizeof stats);
  if (st != AMR_OK) return fail("amr_stats", st);
  st = amr_destroy(ctx);
  if (st != AMR_OK) return fail("amr_destroy", st);
  free(level);
  free(coord);
  free(child);
  free(rho);
  printf("c abi ok: %lld octs, %d x %d pixels, stats %.60s...\n", (long long)n_oct, N, N, stats);
  return 0;
}

/*
 * amr_oracle.c — CPU oracle for the octree ray-casting pass.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously-correct CPU
 * statement of what the ray-casting pass of Sec. 2.2 computes.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg load it; the
 * product library never links, calls or falls back to it, and it shares no
 * source, header or table with the CUDA path.
 *
 * What it computes (Sec. 2.2, Sec. 2, Sec. 2.1 last sentence):
 *   one ray per pixel; every leaf cell the ray crosses contributes its value
 *   times the length between the ray's entry and exit points on the cell faces;
 *   contributions are summed (order-free).  The camera fixes the deepest level
 *   read (Sec. 2): a cell at that level is treated as a leaf.  Modes:
 *     column : S = sum rho_i * len_i
 *     wmean  : sum rho_i * vlos_i * len_i / sum rho_i * len_i   (0 if empty)
 *     max    : max rho_i over crossed leaves (MIP maps, Sec. 2.1)
 *     level  : sum rho_i * len_i * level_i / sum rho_i * len_i, the local mesh
 *              resolution an adaptive blur follows (Sec. 2.2)
 *   and the number of leaves crossed with positive length.
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - cell c of an oct sits at offset (c&1, c>>1&1, c>>2&1); cells are
 *     half-open boxes [k 2^-l, (k+1) 2^-l).
 *   - orthographic camera; pixel (i,j) centre =
 *       centre + ((i+0.5)/nx - 0.5) fov0 u + ((j+0.5)/ny - 0.5) fov1 v,
 *     evaluated in this order in IEEE double without contraction; the ray is
 *     the whole line through it along +w (no near/far cut).
 *   - the ray is quantised: X0 = round-half-even(x 2^36) per axis, direction
 *     D = round-half-even(w / max|w_a| * 2^23).  All decisions are exact
 *     rational comparisons on this quantised line (done here in __int128), so
 *     the set of leaves with positive chord is unique.
 *   - chord = (t_exit - t_entry) * |D|_2 2^-36, t in units where the ray moves
 *     by D per unit.
 *   - max level: a camera max_level > 0 is used as given; max_level < 0 picks
 *     the deepest level whose cell edge is at least one pixel (both axes);
 *     the result is clamped to [1, deepest level of the tree].
 *   - wmean line-of-sight velocity = v . w (w as given, double).
 *
 * Procedure per ray, in the paper's order (Sec. 2.2): find where the ray enters
 * and leaves the box; starting at the entry, descend from the root
 * until a leaf (or a cell at the camera's level) contains the ray; compute the
 * exit point on that cell's faces; add value * length; continue from the exit
 * point with a fresh descent from the root, until the ray leaves the box.
 * Sums are FP64 with Neumaier compensation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef __int128 i128;

enum { OR_OK = 0, OR_E_INVALID = -1, OR_E_BADTREE = -2 };
enum { OR_COLUMN = 0, OR_WMEAN = 1, OR_MAX = 2, OR_LEVEL = 3 };

#define OR_K 36          /* fixed-point bits of a coordinate (level 22 + 14 guard bits) */
#define OR_DBITS 23      /* bits of the largest direction component */

typedef struct {
  double centre[3], u[3], v[3], w[3];
  double fov[2];
  int32_t nx, ny, max_level, mode;
  int32_t field_value, field_weight, field_vel[3];
  int32_t reserved;
} oracle_camera;

/* The quantised ray family of one camera. */
typedef struct {
  int L;              /* deepest level read */
  int64_t D[3];       /* quantised direction */
  int64_t aD[3];      /* |D| */
  double lambda;      /* box length per unit of ray parameter */
} oracle_view;

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static int tree_depth(int64_t n_oct, const uint8_t* level) {
  int d = 1;
  for (int64_t o = 0; o < n_oct; ++o)
    if (level[o] > d) d = level[o];
  return d;
}

/* Camera set-up (Sec. 2: the camera defines the deepest level). */
static int make_view(const oracle_camera* cam, int depth, oracle_view* vw) {
  if (cam->nx <= 0 || cam->ny <= 0) return OR_E_INVALID;
  if (cam->mode < OR_COLUMN || cam->mode > OR_LEVEL) return OR_E_INVALID;
  if (!(cam->fov[0] > 0.0) || !(cam->fov[1] > 0.0)) return OR_E_INVALID;
  const double tol = 1e-9;
  if (fabs(dot3(cam->u, cam->u) - 1.0) > tol || fabs(dot3(cam->v, cam->v) - 1.0) > tol ||
      fabs(dot3(cam->w, cam->w) - 1.0) > tol || fabs(dot3(cam->u, cam->v)) > tol ||
      fabs(dot3(cam->u, cam->w)) > tol || fabs(dot3(cam->v, cam->w)) > tol)
    return OR_E_INVALID;
  int L;
  if (cam->max_level > 0) {
    L = cam->max_level;
  } else {
    /* deepest l with 2^-l >= fov_a / n_a on both axes, i.e. fov_a 2^l <= n_a */
    L = 1;
    for (int l = 1; l <= 22; ++l)
      if (ldexp(cam->fov[0], l) <= (double)cam->nx && ldexp(cam->fov[1], l) <= (double)cam->ny) L = l;
  }
  if (L > depth) L = depth;
  if (L < 1) L = 1;
  vw->L = L;
  double m = fmax(fabs(cam->w[0]), fmax(fabs(cam->w[1]), fabs(cam->w[2])));
  double s2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    vw->D[a] = llrint(ldexp(cam->w[a] / m, OR_DBITS));
    vw->aD[a] = vw->D[a] < 0 ? -vw->D[a] : vw->D[a];
    s2 += (double)vw->D[a] * (double)vw->D[a];
  }
  vw->lambda = ldexp(sqrt(s2), -OR_K);
  return OR_OK;
}

static void pixel_centre(const oracle_camera* cam, int i, int j, double x[3]) {
  double s = (((double)i + 0.5) / (double)cam->nx - 0.5) * cam->fov[0];
  double t = (((double)j + 0.5) / (double)cam->ny - 0.5) * cam->fov[1];
  for (int a = 0; a < 3; ++a) {
    double p = cam->centre[a] + s * cam->u[a];
    x[a] = p + t * cam->v[a];
  }
}

/* The quantised pixel centre X0 = round-half-even(x 2^36); 1 if x leaves [-1, 2]^3. */
static int quantised_origin(const oracle_camera* cam, int i, int j, int64_t X0[3]) {
  double x[3];
  pixel_centre(cam, i, j, x);
  int bad = 0;
  for (int a = 0; a < 3; ++a) {
    if (!(x[a] >= -1.0 && x[a] <= 2.0)) bad = 1;
    X0[a] = bad ? 0 : llrint(ldexp(x[a], OR_K));
  }
  return bad;
}

/* An event: the ray parameter t = num / den with den = |D_axis| > 0. */
typedef struct {
  i128 num, den;
} rtime;

static int time_cmp(rtime a, rtime b) {
  i128 l = a.num * b.den, r = b.num * a.den;
  return (l > r) - (l < r);
}

/* Which side of the plane at fixed-point coordinate M (on axis b) the ray
 * occupies just after time t: 1 = upper (x >= M), 0 = lower. */
static int upper_side_after(const int64_t X0[3], const oracle_view* vw, rtime t, int b, int64_t M) {
  /* position - M at time t, times t.den:  (X0_b - M) den + num D_b */
  i128 sig = ((i128)X0[b] - (i128)M) * t.den + t.num * (i128)vw->D[b];
  if (sig > 0) return 1;
  if (sig < 0) return 0;
  return vw->D[b] >= 0;  /* on the plane: moving up (or staying) -> upper cell */
}

typedef struct {
  double s, c;
} nsum;

static void nadd(nsum* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x))
    a->c += (a->s - t) + x;
  else
    a->c += (x - t) + a->s;
  a->s = t;
}

typedef struct {
  int64_t n_oct;
  const uint8_t* level;
  const int32_t* coord;
  const int32_t* child;
  const double* const* fields;
  int32_t n_fields;
} otree;

/* Mark a cell a ray touched (instrumented pass; marks may be NULL).  Every
 * thread writes the same value, so the relaxed atomic store only keeps the
 * concurrent writes well defined. */
static void mark_cell(uint8_t* marks, int64_t oct, int c) {
  if (marks) __atomic_store_n(&marks[8 * oct + c], (uint8_t)1, __ATOMIC_RELAXED);
}

/* Cast one ray.  Returns OR_OK or OR_E_BADTREE (descent hit an inconsistency).
 * leaf_mark / inner_mark (nullable, [n_oct][8] bytes): set to 1 for every leaf
 * the ray crosses and for every refined cell its descents pass through. */
static int cast_ray(const otree* tr, const oracle_camera* cam, const oracle_view* vw, const int64_t X0[3],
                    double* out, int32_t* count, uint8_t* leaf_mark, uint8_t* inner_mark) {
  const int64_t box = (int64_t)1 << OR_K;
  *out = 0.0;
  *count = 0;
  /* Box entry and exit (Sec. 2.2: intersections between the grid and the ray). */
  rtime tin = {0, 0}, tout = {0, 0};
  int have = 0;
  for (int a = 0; a < 3; ++a) {
    if (vw->D[a] == 0) {
      if (!(X0[a] >= 0 && X0[a] < box)) return OR_OK; /* parallel to the slab, outside it */
      continue;
    }
    rtime en, ex;
    en.den = ex.den = vw->aD[a];
    if (vw->D[a] > 0) {
      en.num = -(i128)X0[a];
      ex.num = (i128)box - X0[a];
    } else {
      en.num = (i128)X0[a] - box;
      ex.num = (i128)X0[a];
    }
    if (!have) {
      tin = en;
      tout = ex;
      have = 1;
    } else {
      if (time_cmp(en, tin) > 0) tin = en;
      if (time_cmp(ex, tout) < 0) tout = ex;
    }
  }
  if (time_cmp(tin, tout) >= 0) return OR_OK; /* misses the box, or touches it with zero length */

  const int weighted = cam->mode == OR_WMEAN || cam->mode == OR_LEVEL;
  const double* rho = tr->fields[weighted ? cam->field_weight : cam->field_value];
  nsum S = {0, 0}, N = {0, 0};
  double M = 0.0;
  int32_t cnt = 0;
  rtime t = tin;
  for (;;) {
    /* Descent from the root to the leaf holding the ray just after t. */
    int64_t oct = 0;
    int lvl = 1;
    int c;
    for (;;) {
      if (tr->level[oct] != lvl) return OR_E_BADTREE;
      c = 0;
      for (int b = 0; b < 3; ++b) {
        int64_t mid = ((int64_t)tr->coord[3 * oct + b] + 1) << (OR_K - lvl);
        c |= upper_side_after(X0, vw, t, b, mid) << b;
      }
      int32_t ch = tr->child[8 * oct + c];
      if (ch < 0 || lvl == vw->L) break;
      if (ch >= tr->n_oct) return OR_E_BADTREE;
      mark_cell(inner_mark, oct, c);
      oct = ch;
      ++lvl;
    }
    /* Exit point of this cell: the earliest face crossing ahead of the ray. */
    int64_t size = (int64_t)1 << (OR_K - lvl);
    rtime texit = {0, 0};
    int have_exit = 0;
    for (int b = 0; b < 3; ++b) {
      if (vw->D[b] == 0) continue;
      int64_t k = (int64_t)tr->coord[3 * oct + b] + ((c >> b) & 1);
      rtime e;
      e.den = vw->aD[b];
      e.num = vw->D[b] > 0 ? (i128)(k + 1) * size - X0[b] : (i128)X0[b] - (i128)k * size;
      if (!have_exit || time_cmp(e, texit) < 0) texit = e;
      have_exit = 1;
    }
    /* Length between entry and exit points. */
    i128 num = texit.num * t.den - t.num * texit.den;
    if (num <= 0) return OR_E_BADTREE; /* cannot happen for a consistent tree */
    double len = (double)num / ((double)texit.den * (double)t.den) * vw->lambda;
    mark_cell(leaf_mark, oct, c);
    double r = rho[8 * oct + c];
    if (cam->mode == OR_COLUMN) {
      nadd(&S, r * len);
    } else if (cam->mode == OR_WMEAN) {
      double vlos = tr->fields[cam->field_vel[0]][8 * oct + c] * cam->w[0] +
                    tr->fields[cam->field_vel[1]][8 * oct + c] * cam->w[1] +
                    tr->fields[cam->field_vel[2]][8 * oct + c] * cam->w[2];
      nadd(&S, r * len);
      nadd(&N, r * vlos * len);
    } else if (cam->mode == OR_LEVEL) {
      nadd(&S, r * len);
      nadd(&N, r * len * (double)lvl);
    } else {
      if (cnt == 0 || r > M) M = r;
    }
    ++cnt;
    if (time_cmp(texit, tout) >= 0) break;
    t = texit;
  }
  if (cam->mode == OR_COLUMN) {
    *out = S.s + S.c;
  } else if (cam->mode == OR_WMEAN || cam->mode == OR_LEVEL) {
    double s = S.s + S.c;
    *out = s != 0.0 ? (N.s + N.c) / s : 0.0;
  } else {
    *out = M;
  }
  *count = cnt;
  return OR_OK;
}

static int field_ok(int32_t f, int32_t n_fields) { return f >= 0 && f < n_fields; }

static int fields_ok(const oracle_camera* cam, int32_t n_fields) {
  if (cam->mode == OR_LEVEL) return field_ok(cam->field_weight, n_fields);
  if (cam->mode != OR_WMEAN) return field_ok(cam->field_value, n_fields);
  return field_ok(cam->field_weight, n_fields) && field_ok(cam->field_vel[0], n_fields) &&
         field_ok(cam->field_vel[1], n_fields) && field_ok(cam->field_vel[2], n_fields);
}

/*
 * Render a camera.  Arrays as produced by the generator (root = oct 0, level 1).
 * fields: n_fields pointers to double[n_oct*8].
 * n_pix < 0: every pixel, map/counts are [ny][nx] row-major, row 0 at -v.
 * n_pix >= 0: only pixels (pix_i[q], pix_j[q]); map/counts have n_pix entries.
 * n_threads: OpenMP threads (0 = runtime default).
 */
int oracle_render(int64_t n_oct, const uint8_t* level, const int32_t* coord, const int32_t* child,
                  int32_t n_fields, const double* const* fields, const oracle_camera* cam, int64_t n_pix,
                  const int32_t* pix_i, const int32_t* pix_j, double* map, int32_t* counts, int32_t n_threads) {
  if (n_oct < 1 || !level || !coord || !child || !fields || !cam || !map || !counts) return OR_E_INVALID;
  if (!fields_ok(cam, n_fields)) return OR_E_INVALID;
  oracle_view vw;
  int st = make_view(cam, tree_depth(n_oct, level), &vw);
  if (st != OR_OK) return st;
  otree tr = {n_oct, level, coord, child, fields, n_fields};
  int64_t total = n_pix >= 0 ? n_pix : (int64_t)cam->nx * cam->ny;
  int err = OR_OK;
#ifdef _OPENMP
  int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
#endif
  for (int64_t q = 0; q < total; ++q) {
    int i = n_pix >= 0 ? pix_i[q] : (int)(q % cam->nx);
    int j = n_pix >= 0 ? pix_j[q] : (int)(q / cam->nx);
    int64_t X0[3];
    int bad = quantised_origin(cam, i, j, X0);
    int s = bad ? OR_E_INVALID : cast_ray(&tr, cam, &vw, X0, &map[q], &counts[q], NULL, NULL);
    if (s != OR_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
      err = s;
    }
  }
  return err;
}

/*
 * Instrumented pass: cast every pixel's ray of the camera (as oracle_render)
 * and mark what it touches: leaf_mark[8 oct + c] = 1 for every leaf crossed
 * (its value is read), inner_mark[8 oct + c] = 1 for every refined cell a
 * descent passes through (its child index is read).  Counting the marks gives
 * the data a frame must read at least once (its compulsory bytes).  Marks are
 * only set, never cleared, so several cameras may accumulate into one array.
 */
int oracle_touched(int64_t n_oct, const uint8_t* level, const int32_t* coord, const int32_t* child,
                   int32_t n_fields, const double* const* fields, const oracle_camera* cam, uint8_t* leaf_mark,
                   uint8_t* inner_mark, int32_t n_threads) {
  if (n_oct < 1 || !level || !coord || !child || !fields || !cam || !leaf_mark || !inner_mark) return OR_E_INVALID;
  if (!fields_ok(cam, n_fields)) return OR_E_INVALID;
  oracle_view vw;
  int st = make_view(cam, tree_depth(n_oct, level), &vw);
  if (st != OR_OK) return st;
  otree tr = {n_oct, level, coord, child, fields, n_fields};
  int64_t total = (int64_t)cam->nx * cam->ny;
  int err = OR_OK;
#ifdef _OPENMP
  int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
#endif
  for (int64_t q = 0; q < total; ++q) {
    int64_t X0[3];
    double v;
    int32_t k;
    int bad = quantised_origin(cam, (int)(q % cam->nx), (int)(q / cam->nx), X0);
    int s = bad ? OR_E_INVALID : cast_ray(&tr, cam, &vw, X0, &v, &k, leaf_mark, inner_mark);
    if (s != OR_OK) {
#ifdef _OPENMP
#pragma omp critical
#endif
      err = s;
    }
  }
  return err;
}

/* The camera's quantised ray family: L, D[3], lambda. */
int oracle_view_info(int64_t n_oct, const uint8_t* level, const oracle_camera* cam, int32_t* L, int64_t* D,
                     double* lambda) {
  oracle_view vw;
  int st = make_view(cam, tree_depth(n_oct, level), &vw);
  if (st != OR_OK) return st;
  *L = vw.L;
  for (int a = 0; a < 3; ++a) D[a] = vw.D[a];
  *lambda = vw.lambda;
  return OR_OK;
}

/* The quantised origin of pixel (i, j): X0[3]. */
int oracle_ray_origin(const oracle_camera* cam, int32_t i, int32_t j, int64_t* X0) {
  return quantised_origin(cam, i, j, X0) ? OR_E_INVALID : OR_OK;
}

/*
 * Slice map (Sec. 3.3, the slice-map tree search): for each pixel centre (on
 * the plane through the camera centre spanned by u and v), the value of the
 * leaf containing that point at the camera's level cut, and that leaf's level
 * (0 and 0 outside the box).  Containment is half-open: the point belongs to
 * the cell whose low faces it lies on.  The descent compares the quantised
 * point with each oct's mid-planes, taken from the coord array.
 */
int oracle_slice(int64_t n_oct, const uint8_t* level, const int32_t* coord, const int32_t* child,
                 int32_t n_fields, const double* const* fields, const oracle_camera* cam, double* map,
                 int32_t* levels, int32_t n_threads) {
  if (n_oct < 1 || !level || !coord || !child || !fields || !cam || !map || !levels) return OR_E_INVALID;
  if (cam->field_value < 0 || cam->field_value >= n_fields) return OR_E_INVALID;
  oracle_view vw;
  int st = make_view(cam, tree_depth(n_oct, level), &vw);
  if (st != OR_OK) return st;
  const int64_t box = (int64_t)1 << OR_K;
  const double* f = fields[cam->field_value];
  int64_t total = (int64_t)cam->nx * cam->ny;
  int err = OR_OK;
#ifdef _OPENMP
  int nt = n_threads > 0 ? n_threads : omp_get_max_threads();
#pragma omp parallel for schedule(static) num_threads(nt)
#endif
  for (int64_t q = 0; q < total; ++q) {
    int64_t X0[3];
    int bad = quantised_origin(cam, (int)(q % cam->nx), (int)(q / cam->nx), X0);
    int inside = 1;
    for (int a = 0; a < 3; ++a)
      if (!(X0[a] >= 0 && X0[a] < box)) inside = 0;
    map[q] = 0.0;
    levels[q] = 0;
    if (bad) {
#ifdef _OPENMP
#pragma omp critical
#endif
      err = OR_E_INVALID;
      continue;
    }
    if (!inside) continue;
    int64_t oct = 0;
    int lvl = 1;
    for (;;) {
      int c = 0;
      for (int b = 0; b < 3; ++b) {
        int64_t mid = ((int64_t)coord[3 * oct + b] + 1) << (OR_K - lvl);
        c |= (X0[b] >= mid) << b;
      }
      int32_t ch = child[8 * oct + c];
      if (ch < 0 || lvl == vw.L) {
        map[q] = f[8 * oct + c];
        levels[q] = lvl;
        break;
      }
      oct = ch;
      ++lvl;
    }
  }
  return err;
}

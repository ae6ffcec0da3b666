/*
 * amr_gen.h — seeded synthetic octree generator (input generation only).
 *
 * Builds RAMSES-style octrees (Sec. 1: an oct holds 8 cells, refinement up to
 * level 22, cells carry scalar and vector fields) in the linearised layout that
 * amr_load_octree() consumes.  It stands in for the Milky-Way simulation
 * outputs of Sec. 1 / Fig. 3, which are not available.  The generator holds none
 * of the ray-casting arithmetic; both the CUDA renderer and the CPU oracle read
 * its arrays.
 *
 * Layout of a generated tree (n_oct octs, breadth-first order, root = 0):
 *   level[n_oct]      uint8   oct level; the root is level 1 (its cells have
 *                             edge 1/2); a cell of level l has edge 2^-l.
 *   coord[n_oct][3]   int32   integer corner of the oct's cell 0, in units of
 *                             level-l cells (always even).
 *   child[n_oct][8]   int32   oct index refining cell c, or -1 (a leaf).
 *                             Cell c sits at offset (c&1, c>>1&1, c>>2&1).
 *   fields[f][n_oct][8]       per-cell values: f = 0 density; f = 1..3 the
 *                             velocity components when with_velocity != 0.
 *                             Refined cells hold restrictions: density = mean
 *                             of the 8 children, velocity = density-weighted
 *                             mean.
 *
 * Ownership: a tree handle owns its arrays until amrgen_free(); amrgen_copy()
 * writes into caller-allocated buffers.  Every function returns 0 on success,
 * a negative code on bad arguments (-1) or allocation failure (-3); none
 * aborts the process.
 */
#ifndef AMR_GEN_H
#define AMR_GEN_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct amrgen_tree amrgen_tree;

enum {
  AMRGEN_PLAIN = 0,   /* rho = 1 + 100 exp(-|x-c|^2 / (2*0.05^2)), absolute mass threshold */
  AMRGEN_GALAXY = 1   /* 1e-6 background + exponential disk x lognormal random field (+ optional Plummer clumps) */
};

typedef struct {
  int32_t kind;           /* AMRGEN_PLAIN or AMRGEN_GALAXY */
  int32_t base_level;     /* every cell of level < base_level is refined */
  int32_t max_level;      /* no cell of level >= max_level is refined (<= 22) */
  int32_t with_velocity;  /* galaxy only: emit 3 velocity fields after density */
  double threshold;       /* refine while rho(centre)*8^-l > threshold (PLAIN: absolute;
                             GALAXY: times the total mass of the base-level grid) */
  uint64_t seed;          /* all random draws (inclination, modes, clumps) */
  int32_t n_modes;        /* Fourier modes per Gaussian random field (GALAXY) */
  int32_t n_clumps;       /* GALAXY: Plummer clumps in the disk, plus one at the centre
                             when > 0 (deep-refinement workload); 0 = none */
  int32_t n_threads;      /* host threads (0 = all) */
  int32_t reserved;
} amrgen_params;

/* Build a tree.  *out receives a handle to free with amrgen_free(). */
int amrgen_build(const amrgen_params* p, amrgen_tree** out);
int64_t amrgen_n_oct(const amrgen_tree* t);
int32_t amrgen_n_fields(const amrgen_tree* t);
/* Copy the arrays out.  fields: n_fields pointers, each [n_oct*8] of
 * float (field_dtype 0) or double (field_dtype 1).  Any pointer may be NULL. */
int amrgen_copy(const amrgen_tree* t, uint8_t* level, int32_t* coord, int32_t* child,
                void* const* fields, int32_t field_dtype);
/* JSON summary: n_oct, n_leaves, leaf histogram per level, total mass, absolute
 * threshold, disk normal.  Returns the length written (truncated to buf_len-1). */
int64_t amrgen_info(const amrgen_tree* t, char* buf, int64_t buf_len);
void amrgen_free(amrgen_tree* t);

/* Evaluate the generator's point functions at n points xyz[n][3]:
 * which = 0 density, 1 the lognormal field g, 2..4 velocity components. */
int amrgen_sample(const amrgen_params* p, int32_t which, int64_t n, const double* xyz, double* out);

#ifdef __cplusplus
}
#endif
#endif

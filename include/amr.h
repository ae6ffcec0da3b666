/*
 * amr.h — C ABI of libamr: octree-AMR volume ray casting on one GB300 GPU.
 *
 * The operation is the ray-casting pass of Sec. 2.2 (the volume ray casting
 * technique): one ray per pixel; each leaf cell the ray crosses contributes its
 * value times the length between the ray's entry and exit points on the cell
 * faces; contributions are added in any order.  The camera fixes the deepest
 * octree level read, so cells at that level act as leaves (Sec. 2, first
 * paragraph).  Besides the column integral the library computes a
 * density-weighted mean of the line-of-sight velocity and the maximum along the
 * ray (maximum-intensity projection, Sec. 2.1 last sentence).
 *
 * Geometry.  The box is the unit cube [0,1)^3.  The root oct has level 1 and
 * its 8 cells have edge 1/2; a cell of level l has edge 2^-l, l <= 22 (Sec. 1:
 * the Milky-Way run is refined to level 22).  Cell c of an oct sits at offset
 * (c&1, c>>1&1, c>>2&1); cells are half-open.  Cameras are orthographic: pixel
 * (i, j) is centred at
 *     centre + ((i+0.5)/nx - 0.5) fov[0] u + ((j+0.5)/ny - 0.5) fov[1] v
 * (IEEE double, in that order, no contraction) and its ray is the whole line
 * through that point along +w.  Map row j = 0 is the -v edge; i runs along +u.
 * The ray is quantised (origin round-half-even(x 2^36) per axis, direction
 * round-half-even(w / max|w_a| 2^23)) and every traversal decision is an exact
 * integer comparison on that line, so the visited-leaf counts are exact.
 *
 * Conventions for every function:
 *   - return AMR_OK (0) or a negative amr_status; never abort the process;
 *   - on error, amr_last_error() returns a message for the calling thread;
 *   - the caller owns every pointer it passes; the library copies what it keeps;
 *   - a context is not thread-safe, except amr_submit / amr_wait / amr_stats,
 *     which may be called from any thread.
 */
#ifndef AMR_H
#define AMR_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct amr_ctx amr_ctx;   /* opaque; owns device memory and streams */
typedef int32_t amr_status;

enum {
  AMR_OK = 0,
  AMR_E_INVALID = -1,    /* bad argument or camera */
  AMR_E_BADTREE = -2,    /* tree arrays fail validation (the oct index is in the message) */
  AMR_E_OOM = -3,        /* device or host allocation failed, or over the memory limit */
  AMR_E_CUDA = -4,       /* a CUDA call failed (its error text is in the message) */
  AMR_E_TIMEOUT = -5,    /* amr_wait ran out of time */
  AMR_E_BUSY = -6,       /* the request queue is full */
  AMR_E_CANCELLED = -7   /* the request was cancelled or the context is shutting down */
};

enum { AMR_F32 = 0, AMR_F64 = 1 };
enum { AMR_MODE_COLUMN = 0, AMR_MODE_WMEAN = 1, AMR_MODE_MAX = 2, AMR_MODE_LEVEL = 3 };
enum { AMR_PREC_FP64 = 0, AMR_PREC_FP32_KAHAN = 1, AMR_PREC_FP32_PLAIN = 2 };
#define AMR_LEVEL_AUTO (-1)   /* deepest level whose cell edge is at least one pixel */

/*
 * A camera (copied at the call).
 *   centre, u, v, w : box units; u, v, w orthonormal to 1e-9; w is the ray direction.
 *   fov             : extent of the map along u and v (orthographic).
 *   nx, ny          : map size in pixels (nx*ny < 2^31).
 *   max_level       : > 0: read levels <= min(max_level, tree depth);
 *                     AMR_LEVEL_AUTO: the deepest level l with 2^-l >= fov[a]/n_a
 *                     on both axes (cells at least one pixel wide, Sec. 2),
 *                     clamped to [1, tree depth].
 *   mode            : AMR_MODE_COLUMN  sum rho*len over crossed leaves
 *                     AMR_MODE_WMEAN   sum rho*(v.w)*len / sum rho*len (0 if empty)
 *                     AMR_MODE_MAX     max rho over crossed leaves (0 if empty)
 *                     AMR_MODE_LEVEL   sum rho*len*level / sum rho*len: the
 *                                      local mesh resolution that amr_blur follows
 *                                      (rho from field_weight; 0 if empty)
 *   precision       : AMR_PREC_FP64 (plain double sums, double map);
 *                     AMR_PREC_FP32_KAHAN (float chords, compensated float sums,
 *                     float map); AMR_PREC_FP32_PLAIN (uncompensated float sums).
 *   field_value     : field used as rho in column and max modes.
 *   field_weight    : field used as rho in wmean mode.
 *   field_vel[3]    : velocity component fields for wmean mode.
 * Every pixel centre must lie in [-1, 2]^3 (it keeps every exact product below
 * 2^62); otherwise AMR_E_INVALID.
 */
typedef struct {
  double centre[3], u[3], v[3], w[3];
  double fov[2];
  int32_t nx, ny, max_level, mode, precision;
  int32_t field_value, field_weight;
  int32_t field_vel[3];
} amr_camera;

/* Launch configuration; chosen by amr_autotune or set by hand. */
typedef struct {
  int32_t tile_w, tile_h;     /* pixels per warp work item: tile_w*tile_h == 32 */
  int32_t block_threads;      /* threads per block: 64..256, multiple of 32 (default 128) */
  int32_t blocks_per_sm;      /* persistent grid = SMs x this (0 = occupancy limit) */
  int32_t tiles_per_grab;     /* work items a warp takes from the queue at once (>= 1) */
  int32_t use_graph;          /* replay batches through a captured CUDA graph */
  int32_t max_regs;           /* registers per thread of the batch kernel: 0 (= 64), 56, 64 or 72;
                                 fewer registers keep more warps resident and spill more.
                                 Partial renders and the no-allocation entry point use 64. */
} amr_options;

/* Create a context on CUDA device `device` (allocates the work queue and a stream). */
amr_status amr_create(amr_ctx** out, int device);
/* Destroy a context: waits for its work, frees all device memory it owns. */
amr_status amr_destroy(amr_ctx* ctx);

/*
 * Load (replace) the octree.  Host arrays, n_oct octs (1 <= n_oct <= (2^31 - 1) / 8,
 * else AMR_E_INVALID: cell indices oct * 8 + c are 32-bit in the kernels):
 *   level[n_oct]        uint8, root = oct 0 at level 1, levels <= 22
 *   coord[n_oct][3]     int32 corner of the oct's cell 0 in level-l cell units (even)
 *   child[n_oct][8]     int32 oct refining cell c, or -1 (leaf)
 *   fields[n_fields]    each [n_oct][8] of float (AMR_F32) or double (AMR_F64)
 * Validation (AMR_E_BADTREE, oct index in the message): root at index 0, level 1,
 * coord 0; child level = parent level + 1; child coord = 2 (parent coord + offset
 * of c); every non-root oct referenced exactly once; coordinates in range.
 * The arrays are renumbered breadth-first (siblings contiguous) into 8-byte oct
 * records {first child, refinement mask | level << 8}, 64-byte link blocks (six
 * face links, each with the linked oct's mask and level, and the packed oct
 * coordinates) and one array per field, and copied to device memory owned by
 * the context (72 B + 8 x field size per oct); the caller may free its arrays
 * on return.
 * Synchronous.
 */
amr_status amr_load_octree(amr_ctx* ctx, int64_t n_oct, const uint8_t* level, const int32_t* coord,
                           const int32_t* child, int32_t n_fields, const void* const* fields,
                           int32_t field_dtype);

/*
 * Render one camera.  map_out: nx*ny values, double for AMR_PREC_FP64 and float
 * otherwise, row-major [ny][nx].  count_out (nullable): nx*ny int32 visited-leaf
 * counts.  out_on_device != 0: both are device pointers and the call returns once
 * the work is enqueued on `cuda_stream` (a cudaStream_t; NULL = the CUDA default
 * stream); out_on_device == 0: host pointers, and the call returns when the
 * results are in them.  Page-locked host buffers that are mapped into the
 * device's address space (cudaHostAlloc, or cudaHostRegister with mapping) are
 * written by the kernel itself over the host link, with no copy afterwards;
 * pageable buffers go through device staging and a copy.
 */
amr_status amr_render(amr_ctx* ctx, const amr_camera* cam, void* map_out, int32_t* count_out,
                      int out_on_device, void* cuda_stream);

/*
 * Render n cameras (uneven sizes, levels, modes) in one persistent launch per
 * precision, fed by a device work queue of ray tiles (Sec. 3.2: a master hands
 * out work to whichever worker is free).  maps[i] / counts[i] as in amr_render;
 * counts may be NULL, and so may any counts[i].
 *
 * Weighted-mean cameras read the weight and the three velocities of a cell as
 * one packed 16-byte word (32 bytes for AMR_F64 fields).  The first render
 * (here, in amr_render or by the server) that uses a given choice of weight and
 * velocity fields builds that packed copy once: it allocates n_oct x 8 x 16 B
 * (x 32 B) of device memory owned by the context and waits for one gather
 * kernel; later renders reuse it, and loading a new tree frees it.  amr_stats
 * reports the copies under tree.packed_fields / tree.packed_bytes.
 */
amr_status amr_render_batch(amr_ctx* ctx, int32_t n, const amr_camera* cams, void* const* maps,
                            int32_t* const* counts, int out_on_device, void* cuda_stream);

/*
 * Slice map (Sec. 3.3: the slice-map tree search the authors moved to the
 * GPU): for each pixel centre — the plane through cam->centre spanned by u, v,
 * the same pixel lattice and quantisation as the rays — the value of
 * cam->field_value in the leaf holding that point at the camera's level cut
 * (half-open cells).  map_out: double [ny][nx] for AMR_PREC_FP64, else float;
 * level_out (nullable): int32 [ny][nx], the level of that leaf, 0 where the
 * point lies outside the box (the value there is 0).  cam->mode is ignored.
 * Pointers and stream as in amr_render.
 */
amr_status amr_slice(amr_ctx* ctx, const amr_camera* cam, void* map_out, int32_t* level_out, int out_on_device,
                     void* cuda_stream);

/*
 * Adaptive Gaussian blur (Sec. 2.2: a post-process whose width follows how
 * finely the mesh is resolved under each pixel, against coarse-cell aliasing).  in, level, out:
 * device float [ny][nx]; level is the AMR_MODE_LEVEL map of the same camera;
 * pixel is the pixel edge in box units (fov[0] / nx).  Per pixel, sigma =
 * 2^-level / (2 pixel) pixels (below 0.5: copied unchanged); separable, rows
 * then columns, each output pixel with its own sigma; weights
 * exp(-k^2 / (2 sigma^2)), |k| <= floor(3 sigma + 0.5) capped at 64, renormalised
 * over the samples inside the map.  in and out may not alias.  Enqueued on
 * cuda_stream; the intermediate buffer belongs to the context (one blur at a
 * time per context).
 */
amr_status amr_blur(amr_ctx* ctx, int32_t nx, int32_t ny, const float* in, const float* level, double pixel,
                    float* out, void* cuda_stream);

/* Validate a camera against the loaded tree; *level_out (nullable) receives the
 * level cut it renders at. */
amr_status amr_camera_check(amr_ctx* ctx, const amr_camera* cam, int32_t* level_out);

amr_status amr_set_options(amr_ctx* ctx, const amr_options* opt);
amr_status amr_get_options(amr_ctx* ctx, amr_options* opt);

/*
 * Time candidate launch configurations on this batch (each run `reps` times,
 * device results discarded) and keep the fastest in the context: the 16 launch
 * shapes (tile 8x4, 4x8, 16x2, 32x1; 128 or 256 threads per block; 1 or 4
 * tiles per queue grab) at the context's register cap, then the other register
 * caps at the best shape.  *best (nullable) receives it; ms_out (nullable) its
 * time.
 */
amr_status amr_autotune(amr_ctx* ctx, int32_t n, const amr_camera* cams, int32_t reps,
                        amr_options* best, double* ms_out);

/*
 * Serving (Sec. 1: iterative interactive zoom).  amr_submit queues a request and
 * returns at once with a ticket.  The server admits queued requests in arrival
 * order while the map-memory budget allows and renders them by continuous
 * batching at tile granularity: each launch takes at most 2^20 rays (whole ray
 * tiles) from the admitted requests, those with the fewest tiles left first,
 * so a request that arrives while others render joins the next launch (about
 * a millisecond away) and small requests overtake large ones; several launch
 * streams (slots) keep the device fed.  A request completes when its last
 * tile lands, and its result goes into the caller's HOST buffers `map` /
 * `counts` (nullable), which must stay valid until amr_wait returns for the
 * ticket: page-locked buffers mapped into the device's address space are
 * written by the kernel in place, others through staging in the server's
 * device arena (one block of the budget's size, allocated at the first
 * submit) and a copy.  amr_wait blocks until the ticket completes or
 * timeout_us elapses (AMR_E_TIMEOUT; the request stays queued; timeout_us < 0
 * waits forever).  amr_server_config sets the slot count (launches in flight,
 * 1..8), the map memory budget in bytes (0 = 1 GiB) and the most requests one
 * launch serves; call it before the first amr_submit.  amr_stats reports
 * latency (arrival to result), queue wait (arrival to the first tile handed
 * to a launch) and render time (from there to the result) as p50 / p99.
 */
amr_status amr_server_config(amr_ctx* ctx, int32_t slots, int64_t map_budget_bytes, int32_t max_batch);
amr_status amr_submit(amr_ctx* ctx, const amr_camera* cam, void* map, int32_t* counts, uint64_t* ticket);
amr_status amr_wait(amr_ctx* ctx, uint64_t ticket, int64_t timeout_us);
amr_status amr_cancel(amr_ctx* ctx, uint64_t ticket);

/*
 * amr_render_batch without any GPU allocation.  The paper has no counterpart:
 * this is for callers that cannot call cudaMalloc, such as a renderer living
 * inside a simulation whose memory manager owns the whole GPU (in-situ
 * visualisation), a latency-critical loop where an allocation could stall on a
 * device-wide synchronisation, or a process held to a fixed memory footprint.
 * It needs no context: the caller passes the tree, the cameras and the outputs,
 * and the launch scratch (camera table, tile prefix sums, work-queue head) lives
 * in a fixed library-owned device array of under 224 KiB that every GPU loading
 * this library holds until exit.
 *   n_oct     1 <= n_oct <= (2^31 - 1) / 8 (AMR_E_INVALID otherwise)
 *   records   device, [n_oct] uint64: bits 0-31 index of the oct's first child
 *             oct, bits 32-39 its refinement mask (bit c set: cell c refined).
 *             Octs breadth-first from the root (index 0, level 1), the children
 *             of an oct contiguous in cell order (the layout amr_load_octree
 *             builds; a breadth-first tree whose siblings are adjacent maps 1:1).
 *   depth     deepest oct level in the tree (1..22).
 *   fields    host array of n_fields device pointers, each [n_oct][8] values of
 *             field_dtype, in the same oct order.
 *   cams, maps, counts, cuda_stream: as in amr_render_batch with device outputs.
 * At most AMR_NOALLOC_MAX_CAMERAS cameras per call; more is AMR_E_INVALID.
 * Runs on the calling thread's current device and returns once enqueued.  The
 * first call on a device looks up the scratch's device address; make that first
 * call before any stream capture.  All calls share the scratch and clear its
 * queue at the start: calls that overlap on the GPU race on it, so order them
 * on one stream.  Record contents are not validated on the host; a child index
 * at or beyond n_oct ends that ray instead of being read, and the kernel records
 * it (and a ray that reaches the step cap) in the scratch's error word, which
 * amr_noalloc_status reports; the call itself has already returned AMR_OK.
 * The scratch's device address is looked up once per device ordinal and kept
 * for the life of the process: do not use this entry point across a
 * cudaDeviceReset or from a CUDA context other than the device's primary one.
 */
#define AMR_NOALLOC_MAX_CAMERAS 256
amr_status amr_render_batch_noalloc(int64_t n_oct, const uint64_t* records, int32_t depth, int32_t n_fields,
                                    const void* const* fields, int32_t field_dtype, int32_t n,
                                    const amr_camera* cams, void* const* maps, int32_t* const* counts,
                                    void* cuda_stream);

/*
 * Device status of the last amr_render_batch_noalloc on the calling thread's
 * current device (the paper has no counterpart).  Synchronises cuda_stream
 * (pass the stream the batch ran on), then writes into caller host memory
 * (each pointer nullable): *host_error 0 (no error), 1 (a child index at or
 * beyond n_oct ended a ray; *host_oct is the oct that held it) or 2 (a ray hit
 * the step cap of 2^25 leaves, which only a corrupted tree reaches);
 * *host_segments the leaves crossed over all rays.  Allocates nothing.
 * AMR_E_INVALID if no no-allocation batch has run on this device.
 */
amr_status amr_noalloc_status(void* cuda_stream, int32_t* host_error, int32_t* host_oct, uint64_t* host_segments);

/*
 * Sort-last rendering (Sec. 3.1: the data is split among processes, each
 * renders its own part, and the partial images are merged; Sec. 2.2: the
 * leaves' contributions are added in any order, so partial sums over disjoint
 * leaf domains add up to the whole ray's sum).
 *
 * amr_render_batch_partial renders like amr_render_batch with device outputs,
 * but stores each pixel's accumulators instead of the finished value, so that
 * renders of disjoint leaf domains (trees whose cells outside the domain hold
 * zero density) can be merged exactly.  partials[i]: device memory, nx*ny
 * elements of
 *                     FP32 precisions                      AMR_PREC_FP64
 *   column            float2 (high, low), value = high+low  double
 *   wmean, level      float4 (S high, S low, N high, N low)  double2 (S, N)
 *   max               float                                  double
 * where S = sum rho*len and N the weighted numerator (sum rho*(v.w)*len, or
 * sum rho*len*level).  counts as in amr_render_batch (per domain: they include
 * the zero-valued cells the domain's tree holds).
 *
 * amr_merge_partials merges n_parts partial maps of one camera (same mode and
 * precision) into the finished map (device, nx*ny floats, or doubles for
 * AMR_PREC_FP64): sums are added with error-free TwoSum transformations and
 * their errors carried in a second accumulator, the weighted mean is N / S
 * (0 where S = 0), and max takes the largest value.  1 <= n_parts <=
 * AMR_MERGE_MAX_PARTS; n_px = nx*ny.  partials is a host array of device
 * pointers.  Runs on the calling thread's current device, enqueued on
 * cuda_stream; allocates nothing.
 */
#define AMR_MERGE_MAX_PARTS 64
amr_status amr_render_batch_partial(amr_ctx* ctx, int32_t n, const amr_camera* cams, void* const* partials,
                                    int32_t* const* counts, void* cuda_stream);
amr_status amr_merge_partials(int32_t n_parts, int32_t mode, int32_t precision, int64_t n_px,
                              const void* const* partials, void* map_out, void* cuda_stream);

/* JSON counters: renders, rays, segments, tree bytes (and the packed
 * weighted-mean copies), options, registers per thread of the batch kernels at
 * the current cap, server latency. */
amr_status amr_stats(amr_ctx* ctx, char* json_buf, int64_t buf_len);

/* Device memory the loaded tree occupies (records, link blocks, fields; the
 * packed weighted-mean copies are counted in amr_stats), its oct count and
 * depth. */
amr_status amr_tree_info(amr_ctx* ctx, int64_t* n_oct, int32_t* depth, int64_t* device_bytes);

/* Message of the calling thread's last error (static storage; ctx may be NULL). */
const char* amr_last_error(amr_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif

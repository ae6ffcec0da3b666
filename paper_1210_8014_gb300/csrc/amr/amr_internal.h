// Internal types shared by the host C ABI (amr_api.cpp) and the CUDA kernels
// (amr_kernels.cu).  Not part of the public interface.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "amr.h"

namespace amr {

constexpr int kFixBits = 36;      // fixed-point bits of a coordinate: level 22 + 14 guard bits
constexpr int kDirBits = 23;      // bits of the largest quantised direction component
constexpr int kMaxLevel = 22;     // deepest level an octree may hold
constexpr int kMaxPrecisions = 3;

// Slot 7 of every link block holds this marker: the increments' link slot for
// a step on several axes at once, which leaves the oct through an edge or a
// corner and is resolved by a descent from the root.
constexpr int32_t kCornerLink = INT32_MIN;

// Error codes a kernel writes into the work-queue block (never traps).
enum : int32_t { kDevOk = 0, kDevBadOct = 1, kDevStepCap = 2 };

// One camera after host canonicalisation: what a warp needs to trace its tile.
struct CamDev {
  double centre[3], u[3], v[3], w[3];
  double fov0, fov1;
  double nxd, nyd;          // nx, ny as doubles (pixel-centre formula)
  double lam;               // box length per unit of ray parameter: |D|_2 2^-36
  double lamInv[3];         // lam / |D_a| (0 where D_a = 0)
  double invD[3];           // 1 / |D_a| (0 where D_a = 0)
  float wF[3];
  // Per (entry axis a, exit axis b), the chord's constants: x = bits of the
  // FP32 factor float(lamInv[a]) * float(invD[b]) (rounded once); K = y + z E
  // with (y, z) = (|D_b| - 1, -1) when a < b, (|D_b|, 1) when a > b and
  // (|D_b|, 0) when a == b; w = index of the remainder part in the per-ray
  // table {r01, s - r01, r02, s - r02, r12, s - r12, 0}: 2 pair + (a < b), or 6
  // when a == b (the time is then s / |D_b| = |D_b| s / (|D_a| |D_b|)).
  int4 chord[3][3];
  // z E by multiply-adds: (x, y, z) = z at the pair's slot of (F01, F02, F12),
  // 0 elsewhere; w = 1 when z = -1.  Then z E = (x F01 + y F02 + z F12 + w) >> 1
  // (F = 2E + [r > 0], so (1 - F) >> 1 = -E).
  int4 chordsel[3][3];
  // For each set of stepped axes (bit a: axis a): x, y, z = increments of the
  // exit-order terms F01, F02, F12 (2|D| per crossed plane); w = face-link slot
  // of the stepped axis, or 7 (the corner marker) when more than one axis steps.
  int4 dF[8];
  // FP64 chord factor for (entry a, exit b): lamInv[a] * invD[b].
  double facD[3][3];
  int32_t D[3];             // quantised direction, |D_a| <= 2^23
  int32_t nx, ny, L, mode;
  int32_t tiles_x;
  int32_t tile0;            // first tile of this camera in the launch (a slice of its tiles)
  const void* rho;          // value field (column, max) or weight field (wmean)
  const void* vel[3];       // wmean velocity fields
  // Weighted mean: (density, v_x, v_y, v_z) of every cell packed into 16
  // bytes (32 for double fields), so a step reads its four values with one
  // load; null when the caller gave separate arrays only.
  const void* pack;
  void* map;                // float* or double* [ny][nx]
  int32_t* counts;          // nullable
  // Pixel-centre terms, [3 (nx + ny)] doubles: (centre + s_i u) 2^36 for each
  // column i, then (t_j v) 2^36 for each row j (s_i, t_j the pixel offsets along
  // u and v), each rounded exactly as the per-ray formula rounds it; filled on
  // the host per launch.  A ray's origin on the 2^-36 lattice is
  // rint(column term + row term).  Null: the kernels evaluate the formula.
  const double* st;
};

// Scratch block one launch owns: queue head, error word, segment counter.
struct QueueBlock {
  int32_t head;
  int32_t error;
  int32_t err_oct;
  int32_t pad;
  unsigned long long segments;
};

struct BatchArgs {
  const uint2* rec;         // oct records {first child, refinement mask | level << 8}
  const int2* nbr;          // [n_oct][8]: six face-neighbour links {target, the
                            // target oct's mask | level << 8}, then the oct's corner
                            // coordinates halved, packed x | y << 21 | z << 42; or
                            // null (then the kernel finds neighbours through its
                            // ancestor stack)
  uint32_t n_oct;
  int32_t n_cams;
  const CamDev* cams;
  const int32_t* tile_start;  // [n_cams + 1] prefix sums of tiles
  int32_t total_tiles;
  int32_t tile_w, tile_h, tiles_per_grab;
  int32_t partial;            // 1: store each pixel's accumulators (a sort-last partial)
  QueueBlock* q;
};

// The loaded tree as camera canonicalisation needs it.
struct TreeView {
  const void* const* fields;  // device pointers, one per field
  int n_fields;
  int depth;                  // deepest oct level present
  bool loaded;
};

// Camera -> CamDev (tile_w: pixels per tile row).  On failure returns
// AMR_E_INVALID and sets the calling thread's amr_last_error() message.
int32_t canonicalise_view(const TreeView& t, const amr_camera& c, int tile_w, CamDev& d);
// Set the calling thread's amr_last_error() message; returns st.
int32_t set_error(int32_t st, const char* msg);

// Register caps per thread of the batch kernel: the default, and the others
// the map-output kernels with links are built with (amr_options.max_regs).
constexpr int kDefaultRegs = 64;
constexpr int kRegCaps[] = {56, 64, 72};
constexpr int kNumRegCaps = 3;
inline int reg_cap_index(int regs) { return regs == 56 ? 0 : (regs == 72 ? 2 : 1); }

// The map-output batch kernel with links at register cap 56 or 72 (as a
// kernel function pointer), or null for another cap.
const void* batch_kernel_capped(int prec, bool f64, int regs);

// Launch one persistent batch kernel.  prec: AMR_PREC_*; f64: field dtype is
// double; regs: register cap (kRegCaps; others mean the default).
cudaError_t launch_batch(int prec, bool f64, const BatchArgs& a, int grid, int block, int regs, cudaStream_t s);
// Slice map of one camera (cam: a device CamDev whose map/counts point to the
// outputs; out64: double map).  err: device int set to 1 on a bad oct index.
cudaError_t launch_slice(bool out64, bool f64, const uint2* rec, uint32_t n_oct, const CamDev* cam, int64_t n_px,
                         int32_t* err, cudaStream_t s);
// Gather four [n_cells] fields into the packed [n_cells][4] array (float or double).
cudaError_t launch_pack(bool f64, const void* f0, const void* f1, const void* f2, const void* f3, void* out,
                        int64_t n_cells, cudaStream_t s);
// Adaptive blur: row pass into tmp, column pass into out (device [ny][nx] floats).
cudaError_t launch_blur(const float* in, const float* level, double pixel, float* tmp, float* out, int nx, int ny,
                        cudaStream_t s);
// Largest resident blocks per SM for the kernel of (prec, f64, with neighbour
// links, register cap) at this block size.
cudaError_t batch_occupancy(int prec, bool f64, bool nb, int block, int regs, int* blocks_per_sm);
// Registers per thread of that kernel (for stats).
int batch_regs(int prec, bool f64, bool nb, int regs);

}  // namespace amr

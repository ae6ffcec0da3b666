// Host side of the libamr C ABI: tree validation and linearisation, camera
// canonicalisation, persistent batch launches, autotuning and the request
// server.  Every path that computes ray results goes through the CUDA kernels
// in amr_kernels.cu; there is no host fallback.
#include "amr.h"
#include "amr_internal.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

using amr::CamDev;
using amr::QueueBlock;

namespace {

thread_local std::string g_err;

amr_status fail(amr_status st, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  std::vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define CUDA_TRY(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) return fail(AMR_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// (density, v_x, v_y, v_z) of every cell packed for one choice of weight and
// velocity fields: the weighted mean's step reads the four with one load.
struct PackedFields {
  int key[4] = {-1, -1, -1, -1};
  void* buf = nullptr;
  int64_t bytes = 0;
};

struct DeviceTree {
  uint2* rec = nullptr;
  std::vector<PackedFields> packs;  // built on first use, freed with the tree
  int2* nbr = nullptr;  // [n_oct][8] 64-byte link blocks: six face links + packed coordinates
  std::vector<void*> fields;
  int64_t n_oct = 0;
  int depth = 0;
  bool f64 = false;
  int64_t bytes = 0;
};

// One launch's scratch in one device block with a pinned host mirror, laid out
// per launch so that all a launch uploads is one contiguous prefix: tile
// prefix sums, queue blocks (zeroed on the host), camera records, pixel-centre
// tables.  One copy uploads it; the queue blocks come back into the mirror.
struct LaunchSlot {
  int cap = 0;                // cameras the tile prefix arrays hold
  char* h_blob = nullptr;     // pinned host mirror
  char* d_blob = nullptr;
  size_t blob_cap = 0;        // bytes of each
  size_t upload = 0;          // bytes the current layout uploads
  // Views of the current layout, host and device.
  int32_t* h_tiles = nullptr;  // kMaxPrecisions x (cap + 1)
  QueueBlock* h_q = nullptr;   // kMaxPrecisions
  CamDev* h_cams = nullptr;
  double* h_st = nullptr;
  int32_t* d_tiles = nullptr;
  QueueBlock* d_q = nullptr;
  CamDev* d_cams = nullptr;
  double* d_st = nullptr;
  cudaEvent_t start = nullptr, done = nullptr;
  bool pending = false;  // a launch whose results are not yet harvested
  int n_groups = 0;
  cudaGraphExec_t gexec = nullptr;  // captured launch sequence of this slot
  std::vector<int64_t> gkey;        // batch shape it was captured for
};

struct Request {
  amr_camera cam;
  void* map = nullptr;
  int32_t* counts = nullptr;
  int64_t bytes = 0;
  amr_status status = AMR_OK;
  int state = 0;  // 0 queued, 1 admitted (its tiles being rendered), 2 done
  std::chrono::steady_clock::time_point t_submit, t_start, t_done;
  std::string err;
  // Tile-granular progress once admitted: the camera with its output pointers
  // (the caller's page-locked buffers, or staging in the server arena), its
  // tiles, how many are handed to launches, how many are finished.
  CamDev dev;
  int64_t tiles = 0, next = 0, finished = 0;
  int64_t stage_off = -1;  // arena offset of the staging, or -1 (written in place)
  bool failed = false;
};

struct ServerSlot {
  cudaStream_t stream = nullptr;
  std::thread th;
};

// First-fit allocator over one device block (the server's map-memory arena):
// staging for requests whose host buffers the GPU cannot write directly.
struct Arena {
  char* base = nullptr;
  int64_t size = 0;
  std::map<int64_t, int64_t> free;  // offset -> bytes, coalesced
  void reset(int64_t n) {
    size = n;
    free.clear();
    if (n > 0) free[0] = n;
  }
  int64_t take(int64_t n) {
    n = (n + 255) / 256 * 256;
    for (auto it = free.begin(); it != free.end(); ++it) {
      if (it->second < n) continue;
      const int64_t off = it->first, rest = it->second - n;
      free.erase(it);
      if (rest) free[off + n] = rest;
      return off;
    }
    return -1;
  }
  void give(int64_t off, int64_t n) {
    n = (n + 255) / 256 * 256;
    auto it = free.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free.erase(nx);
    }
    if (it != free.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free.erase(it);
      }
    }
  }
};

}  // namespace

struct amr_ctx {
  int device = 0;
  int sms = 0;
  cudaStream_t stream = nullptr;
  DeviceTree tree;
  amr_options opt{8, 4, 128, 0, 1, 0, 0};
  std::mutex launch_mu;  // guards slots and stats
  std::mutex pack_mu;    // guards tree.packs
  std::vector<LaunchSlot> slots;
  size_t next_slot = 0;
  void* blur_tmp = nullptr;  // intermediate of the separable blur
  int64_t blur_cap = 0;
  void* stage = nullptr;  // device staging for host-output renders
  int64_t stage_cap = 0;
  // stats
  int64_t n_renders = 0, n_cams = 0, n_rays = 0;
  int64_t n_h2d_bytes = 0;  // camera tables, tile prefix sums and offset tables uploaded
  unsigned long long n_segments = 0;
  int64_t n_dev_errors = 0;
  double last_batch_ms = 0.0;
  double autotune_ms = -1.0;
  int64_t n_graph_captures = 0, n_graph_launches = 0;
  // resident blocks per SM, by precision, dtype, register cap, block/32
  int occupancy[amr::kMaxPrecisions][2][amr::kNumRegCaps][33] = {};
  // server
  std::mutex srv_mu;
  std::condition_variable srv_cv;   // work arrived / budget freed / stop
  std::condition_variable done_cv;  // a request finished
  std::map<uint64_t, std::shared_ptr<Request>> reqs;
  std::deque<std::shared_ptr<Request>> queue;      // submitted, not yet admitted
  std::vector<std::shared_ptr<Request>> active;    // admitted, tiles outstanding
  Arena arena;
  amr_options srv_opt{};                            // launch options of every server launch
  uint64_t next_ticket = 1;
  int srv_slots = 2;
  int64_t srv_budget = int64_t(1) << 30;
  int64_t srv_used = 0;
  int srv_max_batch = 64;
  int srv_max_queue = 1 << 16;
  bool srv_started = false;
  bool srv_stop = false;
  std::vector<std::unique_ptr<ServerSlot>> srv;
  std::vector<double> latencies_ms, waits_ms, services_ms;  // arrival->result, arrival->admission, admission->result
  int64_t srv_batches = 0, srv_done = 0, srv_failed = 0, srv_max_inflight = 0, srv_inflight = 0;
  std::chrono::steady_clock::time_point srv_t0, srv_tlast;
};

namespace {

constexpr int kSlots = 8;

void free_slot(LaunchSlot& s) {
  if (s.gexec) cudaGraphExecDestroy(s.gexec);
  if (s.h_blob) cudaFreeHost(s.h_blob);
  if (s.d_blob) cudaFree(s.d_blob);
  s = LaunchSlot{};
}

// Lay the slot out for n cameras and st_doubles of pixel-centre tables,
// growing the block when it is too small (a graph captured against the old
// block is dropped), and zero the queue blocks in the host mirror.
amr_status layout_slot(LaunchSlot& s, int n, int64_t st_doubles) {
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  const int cap = s.cap >= n ? s.cap : std::max(n, std::max(64, s.cap * 2));
  const size_t T = up((size_t)amr::kMaxPrecisions * (cap + 1) * sizeof(int32_t));
  const size_t Q = up(amr::kMaxPrecisions * sizeof(QueueBlock));
  const size_t C = up((size_t)n * sizeof(CamDev));
  const size_t total = T + Q + C + (size_t)st_doubles * sizeof(double);
  if (!s.h_blob || s.blob_cap < total) {
    if (s.gexec) cudaGraphExecDestroy(s.gexec);
    s.gexec = nullptr;
    s.gkey.clear();
    if (s.h_blob) cudaFreeHost(s.h_blob);
    if (s.d_blob) cudaFree(s.d_blob);
    s.h_blob = nullptr;
    s.d_blob = nullptr;
    s.blob_cap = 0;
    const size_t want = std::max(total, std::max<size_t>(size_t(1) << 20, 2 * s.blob_cap));
    if (cudaMallocHost((void**)&s.h_blob, want) != cudaSuccess || cudaMalloc((void**)&s.d_blob, want) != cudaSuccess) {
      cudaGetLastError();
      if (s.h_blob) cudaFreeHost(s.h_blob);
      s.h_blob = nullptr;
      s.d_blob = nullptr;
      s.cap = 0;
      return fail(AMR_E_OOM, "cannot allocate %zu bytes of launch scratch", want);
    }
    s.blob_cap = want;
  }
  s.cap = cap;
  s.upload = total;
  s.h_tiles = (int32_t*)s.h_blob;
  s.d_tiles = (int32_t*)s.d_blob;
  s.h_q = (QueueBlock*)(s.h_blob + T);
  s.d_q = (QueueBlock*)(s.d_blob + T);
  s.h_cams = (CamDev*)(s.h_blob + T + Q);
  s.d_cams = (CamDev*)(s.d_blob + T + Q);
  s.h_st = (double*)(s.h_blob + T + Q + C);
  s.d_st = (double*)(s.d_blob + T + Q + C);
  std::memset(s.h_q, 0, Q);
  return AMR_OK;
}

// The pixel-centre terms of one camera, in IEEE double with exactly the
// operations (and order) of the per-ray formula x = (centre + s_i u) + t_j v,
// s_i = ((i + 0.5) / nx - 0.5) fov0, t_j = ((j + 0.5) / ny - 0.5) fov1.  A
// column of rays shares centre + s_i u and a row t_j v, so the table holds
// those, already times 2^36 (exact: a power of two), 3 doubles per column then
// 3 per row; a ray's lattice origin is then rint(A_i + B_j) per axis, the same
// single rounding of the same two operands as the formula.
void pixel_offsets(const CamDev& c, double* out) {
  for (int i = 0; i < c.nx; ++i) {
    const double s = (((double)i + 0.5) / c.nxd - 0.5) * c.fov0;
    for (int a = 0; a < 3; ++a) out[3 * i + a] = (c.centre[a] + s * c.u[a]) * 68719476736.0;
  }
  double* row = out + 3 * (size_t)c.nx;
  for (int j = 0; j < c.ny; ++j) {
    const double t = (((double)j + 0.5) / c.nyd - 0.5) * c.fov1;
    for (int a = 0; a < 3; ++a) row[3 * j + a] = (t * c.v[a]) * 68719476736.0;
  }
}

// Doubles of pixel-centre tables a camera needs.
int64_t offset_doubles(const CamDev& c) { return 3 * ((int64_t)c.nx + c.ny); }

// Fill the slot's pixel-centre tables for its first n cameras (laid out for
// them) and point the camera records there.
void fill_offsets(LaunchSlot& s, int n) {
  int64_t o = 0;
  for (int i = 0; i < n; ++i) {
    CamDev& c = s.h_cams[i];
    pixel_offsets(c, s.h_st + o);
    c.st = s.d_st + o;
    o += offset_doubles(c);
  }
}

amr_status init_slots(amr_ctx* ctx) {
  ctx->slots.resize(kSlots);
  for (auto& s : ctx->slots) {
    CUDA_TRY(cudaEventCreate(&s.start));
    CUDA_TRY(cudaEventCreate(&s.done));
    amr_status st = layout_slot(s, 64, 0);
    if (st != AMR_OK) return st;
  }
  return AMR_OK;
}

// Fold a finished launch's counters into the context (launch_mu held).
amr_status harvest(amr_ctx* ctx, LaunchSlot& s) {
  if (!s.pending) return AMR_OK;
  s.pending = false;
  float ms = 0.0f;
  if (cudaEventElapsedTime(&ms, s.start, s.done) == cudaSuccess) ctx->last_batch_ms = ms;
  else cudaGetLastError();
  amr_status st = AMR_OK;
  for (int g = 0; g < s.n_groups; ++g) {
    ctx->n_segments += s.h_q[g].segments;
    if (s.h_q[g].error != amr::kDevOk) {
      ctx->n_dev_errors++;
      st = fail(AMR_E_CUDA, "kernel reported error %d (oct %d)", s.h_q[g].error, s.h_q[g].err_oct);
    }
  }
  return st;
}

double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

bool finite3(const double* a) { return std::isfinite(a[0]) && std::isfinite(a[1]) && std::isfinite(a[2]); }

// Pixel centre as the kernels compute it (host compiled without contraction).
void pixel_centre(const amr_camera& c, int i, int j, double x[3]) {
  double s = (((double)i + 0.5) / (double)c.nx - 0.5) * c.fov[0];
  double t = (((double)j + 0.5) / (double)c.ny - 0.5) * c.fov[1];
  for (int a = 0; a < 3; ++a) {
    double p = c.centre[a] + s * c.u[a];
    x[a] = p + t * c.v[a];
  }
}

// Camera -> the constants its rays need (Sec. 2: the camera fixes the deepest
// level read).  Returns AMR_E_INVALID with a message on a bad camera.
amr_status canonicalise_tree(const amr::TreeView& t, const amr_camera& c, int tile_w, CamDev& d) {
  if (!t.loaded) return fail(AMR_E_INVALID, "no octree loaded");
  if (c.nx <= 0 || c.ny <= 0 || (int64_t)c.nx * c.ny >= (int64_t(1) << 31))
    return fail(AMR_E_INVALID, "map size %d x %d out of range", c.nx, c.ny);
  if (c.mode < AMR_MODE_COLUMN || c.mode > AMR_MODE_LEVEL) return fail(AMR_E_INVALID, "unknown mode %d", c.mode);
  if (c.precision < AMR_PREC_FP64 || c.precision > AMR_PREC_FP32_PLAIN)
    return fail(AMR_E_INVALID, "unknown precision %d", c.precision);
  d.pack = nullptr;
  const int nf = t.n_fields;
  auto fok = [nf](int f) { return f >= 0 && f < nf; };
  if (c.mode == AMR_MODE_WMEAN) {
    if (!fok(c.field_weight) || !fok(c.field_vel[0]) || !fok(c.field_vel[1]) || !fok(c.field_vel[2]))
      return fail(AMR_E_INVALID, "wmean needs a weight field and 3 velocity fields (tree has %d fields)", nf);
  } else if (c.mode == AMR_MODE_LEVEL) {
    if (!fok(c.field_weight)) return fail(AMR_E_INVALID, "weight field %d out of range", c.field_weight);
  } else if (!fok(c.field_value)) {
    return fail(AMR_E_INVALID, "field %d out of range (tree has %d fields)", c.field_value, nf);
  }
  if (!finite3(c.centre) || !finite3(c.u) || !finite3(c.v) || !finite3(c.w) || !std::isfinite(c.fov[0]) ||
      !std::isfinite(c.fov[1]) || !(c.fov[0] > 0.0) || !(c.fov[1] > 0.0))
    return fail(AMR_E_INVALID, "camera has a non-finite value or a non-positive field of view");
  const double tol = 1e-9;
  if (std::fabs(dot3(c.u, c.u) - 1.0) > tol || std::fabs(dot3(c.v, c.v) - 1.0) > tol ||
      std::fabs(dot3(c.w, c.w) - 1.0) > tol || std::fabs(dot3(c.u, c.v)) > tol || std::fabs(dot3(c.u, c.w)) > tol ||
      std::fabs(dot3(c.v, c.w)) > tol)
    return fail(AMR_E_INVALID, "camera axes u, v, w are not orthonormal to 1e-9");
  int L;
  if (c.max_level > 0) {
    L = c.max_level;
  } else if (c.max_level == AMR_LEVEL_AUTO) {
    // deepest l with 2^-l >= fov_a / n_a, i.e. fov_a * 2^l <= n_a (exact in double)
    L = 1;
    while (L < amr::kMaxLevel && std::ldexp(c.fov[0], L + 1) <= (double)c.nx &&
           std::ldexp(c.fov[1], L + 1) <= (double)c.ny)
      ++L;
  } else {
    return fail(AMR_E_INVALID, "max_level %d: use > 0 or AMR_LEVEL_AUTO", c.max_level);
  }
  L = std::max(1, std::min(L, t.depth));
  // The four corner pixels bound every pixel centre (the formula is monotone in i and j).
  const int ci[2] = {0, c.nx - 1}, cj[2] = {0, c.ny - 1};
  for (int p = 0; p < 2; ++p)
    for (int q = 0; q < 2; ++q) {
      double x[3];
      pixel_centre(c, ci[p], cj[q], x);
      for (int a = 0; a < 3; ++a)
        if (!(x[a] >= -1.0 && x[a] <= 2.0))
          return fail(AMR_E_INVALID, "pixel centres leave [-1, 2]^3 (axis %d: %.17g)", a, x[a]);
    }
  std::memset(&d, 0, sizeof d);
  const double wm = std::fmax(std::fabs(c.w[0]), std::fmax(std::fabs(c.w[1]), std::fabs(c.w[2])));
  double s2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    long long q = std::llrint(std::ldexp(c.w[a] / wm, amr::kDirBits));
    d.D[a] = (int32_t)q;
    s2 += (double)q * (double)q;
  }
  d.lam = std::ldexp(std::sqrt(s2), -amr::kFixBits);
  float lamInvF[3], invDF[3];
  for (int a = 0; a < 3; ++a) {
    const double ad = std::fabs((double)d.D[a]);
    d.invD[a] = ad > 0 ? 1.0 / ad : 0.0;
    d.lamInv[a] = ad > 0 ? d.lam / ad : 0.0;
    invDF[a] = (float)d.invD[a];
    lamInvF[a] = (float)d.lamInv[a];
    d.centre[a] = c.centre[a];
    d.u[a] = c.u[a];
    d.v[a] = c.v[a];
    d.w[a] = c.w[a];
    d.wF[a] = (float)c.w[a];
  }
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      const float fac = lamInvF[a] * invDF[b];
      std::memcpy(&d.chord[a][b].x, &fac, sizeof fac);
      const int32_t adb = d.D[b] < 0 ? -d.D[b] : d.D[b];
      d.chord[a][b].y = a < b ? adb - 1 : adb;
      d.chord[a][b].z = a == b ? 0 : (a < b ? -1 : 1);
      d.chord[a][b].w = a == b ? 6 : 2 * (a + b - 1) + (a < b ? 1 : 0);
      int sel[3] = {0, 0, 0};
      if (a != b) sel[a + b - 1] = d.chord[a][b].z;
      d.chordsel[a][b] = make_int4(sel[0], sel[1], sel[2], d.chord[a][b].z < 0 ? 1 : 0);
      d.facD[a][b] = d.lamInv[a] * d.invD[b];
    }
  {
    const int32_t A0 = 2 * std::abs(d.D[0]), A1 = 2 * std::abs(d.D[1]), A2 = 2 * std::abs(d.D[2]);
    for (int sb = 0; sb < 8; ++sb) {
      int32_t x = 0, y = 0, z = 0;
      if (sb & 1) { x += A1; y += A2; }
      if (sb & 2) { x -= A0; z += A2; }
      if (sb & 4) { y -= A0; z -= A1; }
      // w: the face-link slot of the stepped axis b (2b when the ray moves
      // down b, 2b + 1 when it moves up), or 7 (the corner marker) when
      // several axes step.
      int w = 0;
      if (sb) {
        const int b = (sb & 1) ? 0 : ((sb & 2) ? 1 : 2);
        w = 2 * b + (d.D[b] < 0 ? 0 : 1);
        if (sb & (sb - 1)) w = 7;
      }
      d.dF[sb] = make_int4(x, y, z, w);
    }
  }
  d.fov0 = c.fov[0];
  d.fov1 = c.fov[1];
  d.nxd = (double)c.nx;
  d.nyd = (double)c.ny;
  d.nx = c.nx;
  d.ny = c.ny;
  d.L = L;
  d.mode = c.mode;
  d.tiles_x = (c.nx + tile_w - 1) / tile_w;
  if (c.mode == AMR_MODE_WMEAN) {
    d.rho = t.fields[c.field_weight];
    for (int a = 0; a < 3; ++a) d.vel[a] = t.fields[c.field_vel[a]];
  } else if (c.mode == AMR_MODE_LEVEL) {
    d.rho = t.fields[c.field_weight];
  } else {
    d.rho = t.fields[c.field_value];
  }
  return AMR_OK;
}

amr_status canonicalise(const amr_ctx* ctx, const amr_camera& c, int tile_w, int tile_h, CamDev& d) {
  (void)tile_h;
  const DeviceTree& t = ctx->tree;
  const amr::TreeView view{t.fields.data(), (int)t.fields.size(), t.depth, t.rec != nullptr};
  return canonicalise_tree(view, c, tile_w, d);
}

// A weighted-mean camera reads (density, v_x, v_y, v_z) packed per cell: find
// the packed array of its fields, or build it (one gather kernel on a stream of
// its own, waited for, so every later launch on any stream sees it).
amr_status attach_pack(amr_ctx* ctx, const amr_camera& c, CamDev& d) {
  if (c.mode != AMR_MODE_WMEAN) return AMR_OK;
  const int key[4] = {c.field_weight, c.field_vel[0], c.field_vel[1], c.field_vel[2]};
  std::lock_guard<std::mutex> lk(ctx->pack_mu);
  DeviceTree& t = ctx->tree;
  for (const PackedFields& p : t.packs)
    if (std::equal(key, key + 4, p.key)) {
      d.pack = p.buf;
      return AMR_OK;
    }
  const int64_t cells = t.n_oct * 8;
  PackedFields p;
  p.bytes = cells * 4 * (t.f64 ? 8 : 4);
  if (cudaMalloc(&p.buf, (size_t)p.bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(AMR_E_OOM, "cannot allocate %lld bytes of packed weighted-mean fields", (long long)p.bytes);
  }
  cudaStream_t s = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess)
    e = amr::launch_pack(t.f64, t.fields[key[0]], t.fields[key[1]], t.fields[key[2]], t.fields[key[3]], p.buf, cells, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (s) cudaStreamDestroy(s);
  if (e != cudaSuccess) {
    cudaFree(p.buf);
    return fail(AMR_E_CUDA, "packing weighted-mean fields: %s", cudaGetErrorString(e));
  }
  std::copy(key, key + 4, p.key);
  t.packs.push_back(p);
  d.pack = p.buf;
  return AMR_OK;
}

int64_t tiles_of(const CamDev& d, int tile_w, int tile_h) {
  return (int64_t)((d.nx + tile_w - 1) / tile_w) * ((d.ny + tile_h - 1) / tile_h);
}

int64_t map_bytes(const amr_camera& c) {
  return (int64_t)c.nx * c.ny * (c.precision == AMR_PREC_FP64 ? 8 : 4);
}

amr_status check_options(const amr_options& o) {
  if (o.tile_w < 1 || o.tile_h < 1 || o.tile_w * o.tile_h != 32)
    return fail(AMR_E_INVALID, "tile %d x %d: tile_w * tile_h must be 32", o.tile_w, o.tile_h);
  if (o.block_threads < 64 || o.block_threads > 256 || o.block_threads % 32)
    return fail(AMR_E_INVALID, "block_threads %d: use 64..256, a multiple of 32", o.block_threads);
  if (o.blocks_per_sm < 0 || o.blocks_per_sm > 32) return fail(AMR_E_INVALID, "blocks_per_sm %d", o.blocks_per_sm);
  if (o.tiles_per_grab < 1 || o.tiles_per_grab > 64) return fail(AMR_E_INVALID, "tiles_per_grab %d", o.tiles_per_grab);
  if (o.max_regs != 0 && o.max_regs != 56 && o.max_regs != 64 && o.max_regs != 72)
    return fail(AMR_E_INVALID, "max_regs %d: use 0 (the default, 64), 56, 64 or 72", o.max_regs);
  return AMR_OK;
}

// Enqueue one batch of canonical cameras (map/count pointers already device
// pointers) on `stream`: one persistent launch per precision present.
// tiles (nullable): per camera, the number of tiles to render starting at its
// tile0 (a slice of the camera); null renders every camera whole.
amr_status enqueue(amr_ctx* ctx, const amr_options& opt, const std::vector<CamDev>& cams,
                   const std::vector<int>& precs, cudaStream_t stream, LaunchSlot** used, bool partial = false,
                   const std::vector<int64_t>* tiles = nullptr) {
  std::unique_lock<std::mutex> lk(ctx->launch_mu);
  LaunchSlot& s = ctx->slots[ctx->next_slot];
  ctx->next_slot = (ctx->next_slot + 1) % ctx->slots.size();
  if (s.pending) {
    CUDA_TRY(cudaEventSynchronize(s.done));
    harvest(ctx, s);
  }
  const int n = (int)cams.size();
  int64_t st_total = 0;
  for (const CamDev& c : cams) st_total += offset_doubles(c);
  amr_status st = layout_slot(s, n, st_total);
  if (st != AMR_OK) return st;
  // Order cameras by precision group; each group gets its own prefix table.
  int groups[amr::kMaxPrecisions] = {0, 0, 0};
  int gstart[amr::kMaxPrecisions + 1] = {0, 0, 0, 0};
  for (int p : precs) groups[p]++;
  for (int g = 0; g < amr::kMaxPrecisions; ++g) gstart[g + 1] = gstart[g] + groups[g];
  int fill[amr::kMaxPrecisions] = {gstart[0], gstart[1], gstart[2]};
  std::vector<int64_t> ntiles(n);
  for (int i = 0; i < n; ++i) {
    const int k = fill[precs[i]]++;
    s.h_cams[k] = cams[i];
    ntiles[k] = tiles ? (*tiles)[i] : tiles_of(cams[i], opt.tile_w, opt.tile_h);
  }
  fill_offsets(s, n);
  int64_t tiles_total[amr::kMaxPrecisions] = {0, 0, 0};
  for (int g = 0; g < amr::kMaxPrecisions; ++g) {
    int32_t* tp = s.h_tiles + (size_t)g * (s.cap + 1);
    int64_t acc = 0;
    for (int i = 0; i < groups[g]; ++i) {
      tp[i] = (int32_t)acc;
      acc += ntiles[gstart[g] + i];
    }
    tp[groups[g]] = (int32_t)acc;
    if (acc >= (int64_t(1) << 31) - 4096) return fail(AMR_E_INVALID, "batch too large: %lld tiles", (long long)acc);
    tiles_total[g] = acc;
  }
  // Launch plan: one persistent launch per precision group present.  Partial
  // renders keep the default register cap.
  const int regs = partial || opt.max_regs == 0 ? amr::kDefaultRegs : opt.max_regs;
  amr::BatchArgs args[amr::kMaxPrecisions];
  int grids[amr::kMaxPrecisions] = {0, 0, 0};
  for (int g = 0; g < amr::kMaxPrecisions; ++g) {
    if (!groups[g] || !tiles_total[g]) continue;
    amr::BatchArgs& a = args[g];
    a = amr::BatchArgs{};
    a.rec = ctx->tree.rec;
    a.nbr = ctx->tree.nbr;
    a.n_oct = (uint32_t)ctx->tree.n_oct;
    a.n_cams = groups[g];
    a.cams = s.d_cams + gstart[g];
    a.tile_start = s.d_tiles + (size_t)g * (s.cap + 1);
    a.total_tiles = (int32_t)tiles_total[g];
    a.tile_w = opt.tile_w;
    a.tile_h = opt.tile_h;
    a.tiles_per_grab = opt.tiles_per_grab;
    a.partial = partial ? 1 : 0;
    a.q = s.d_q + g;
    int bps = opt.blocks_per_sm;
    if (bps <= 0) {
      int& cached = ctx->occupancy[g][ctx->tree.f64 ? 1 : 0][amr::reg_cap_index(regs)][opt.block_threads / 32];
      if (cached <= 0) CUDA_TRY(amr::batch_occupancy(g, ctx->tree.f64, true, opt.block_threads, regs, &cached));
      bps = std::max(1, cached);
    }
    int64_t grid = (int64_t)ctx->sms * bps;
    const int64_t warps_needed = (tiles_total[g] + opt.tiles_per_grab - 1) / opt.tiles_per_grab;
    const int64_t blocks_needed = (warps_needed * 32 + opt.block_threads - 1) / opt.block_threads;
    grids[g] = (int)std::max<int64_t>(1, std::min(grid, blocks_needed));
  }
  // In a capture the two events must become event-record nodes of the graph
  // (external records), not capture-internal dependencies.
  auto record = [&](cudaStream_t st, bool capturing) -> cudaError_t {
    const unsigned ev = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    cudaError_t e = cudaEventRecordWithFlags(s.start, st, ev);
    // one upload: tile prefix sums, zeroed queue blocks, cameras, pixel tables
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.d_blob, s.h_blob, s.upload, cudaMemcpyHostToDevice, st);
    for (int g = 0; g < amr::kMaxPrecisions && e == cudaSuccess; ++g)
      if (grids[g]) e = amr::launch_batch(g, ctx->tree.f64, args[g], grids[g], opt.block_threads, regs, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s.h_q, s.d_q, amr::kMaxPrecisions * sizeof(QueueBlock), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(s.done, st, ev);
    return e;
  };
  s.n_groups = amr::kMaxPrecisions;
  if (opt.use_graph) {
    // Replay a captured graph of this slot when the batch shape is unchanged
    // (the camera table itself is read from the slot's pinned staging).
    std::vector<int64_t> key = {n, partial ? 1 : 0, s.cap, (int64_t)(uintptr_t)s.d_cams, st_total, (int64_t)(uintptr_t)s.d_st,
                                (int64_t)(uintptr_t)ctx->tree.rec,
                                (int64_t)(uintptr_t)ctx->tree.nbr, ctx->tree.f64, opt.block_threads,
                                opt.tile_w, opt.tile_h, opt.tiles_per_grab, regs};
    for (int g = 0; g < amr::kMaxPrecisions; ++g) {
      key.push_back(groups[g]);
      key.push_back(tiles_total[g]);
      key.push_back(grids[g]);
    }
    if (!s.gexec || s.gkey != key) {
      if (s.gexec) cudaGraphExecDestroy(s.gexec);
      s.gexec = nullptr;
      CUDA_TRY(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = record(ctx->stream, true);
      cudaGraph_t graph = nullptr;
      cudaError_t e2 = cudaStreamEndCapture(ctx->stream, &graph);
      if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return fail(AMR_E_CUDA, "graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
      }
      e = cudaGraphInstantiate(&s.gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        s.gexec = nullptr;
        return fail(AMR_E_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
      }
      s.gkey = key;
      ctx->n_graph_captures++;
    }
    CUDA_TRY(cudaGraphLaunch(s.gexec, stream));
    ctx->n_graph_launches++;
  } else {
    CUDA_TRY(record(stream, false));
  }
  s.pending = true;
  ctx->n_renders++;
  ctx->n_cams += n;
  ctx->n_h2d_bytes += (int64_t)s.upload;
  for (int i = 0; i < n; ++i)
    ctx->n_rays += tiles ? (*tiles)[i] * opt.tile_w * opt.tile_h : (int64_t)cams[i].nx * cams[i].ny;
  if (used) *used = &s;
  return AMR_OK;
}

// One slice-map launch through a launch slot (the camera record and error word
// live in the slot's scratch, so back-to-back calls on any stream do not race).
amr_status enqueue_slice(amr_ctx* ctx, const CamDev& cam, bool out64, cudaStream_t stream, LaunchSlot** used) {
  std::unique_lock<std::mutex> lk(ctx->launch_mu);
  LaunchSlot& s = ctx->slots[ctx->next_slot];
  ctx->next_slot = (ctx->next_slot + 1) % ctx->slots.size();
  if (s.pending) {
    CUDA_TRY(cudaEventSynchronize(s.done));
    harvest(ctx, s);
  }
  amr_status st = layout_slot(s, 1, offset_doubles(cam));
  if (st != AMR_OK) return st;
  s.h_cams[0] = cam;
  fill_offsets(s, 1);
  s.n_groups = amr::kMaxPrecisions;
  CUDA_TRY(cudaEventRecord(s.start, stream));
  CUDA_TRY(cudaMemcpyAsync(s.d_blob, s.h_blob, s.upload, cudaMemcpyHostToDevice, stream));
  ctx->n_h2d_bytes += (int64_t)s.upload;
  CUDA_TRY(amr::launch_slice(out64, ctx->tree.f64, ctx->tree.rec, (uint32_t)ctx->tree.n_oct, s.d_cams,
                             (int64_t)cam.nx * cam.ny, &s.d_q[0].error, stream));
  CUDA_TRY(cudaMemcpyAsync(s.h_q, s.d_q, amr::kMaxPrecisions * sizeof(QueueBlock), cudaMemcpyDeviceToHost, stream));
  CUDA_TRY(cudaEventRecord(s.done, stream));
  s.pending = true;
  ctx->n_renders++;
  if (used) *used = &s;
  return AMR_OK;
}

amr_status finish_sync(amr_ctx* ctx, LaunchSlot* s) {
  CUDA_TRY(cudaEventSynchronize(s->done));
  std::lock_guard<std::mutex> lk(ctx->launch_mu);
  return harvest(ctx, *s);
}

amr_status ensure_stage(amr_ctx* ctx, int64_t bytes) {
  if (ctx->stage_cap >= bytes) return AMR_OK;
  if (ctx->stage) cudaFree(ctx->stage);
  ctx->stage = nullptr;
  ctx->stage_cap = 0;
  if (cudaMalloc(&ctx->stage, (size_t)bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(AMR_E_OOM, "cannot allocate %lld bytes of output staging", (long long)bytes);
  }
  ctx->stage_cap = bytes;
  return AMR_OK;
}

// Device address of a host buffer the GPU can write directly: page-locked
// memory mapped into the device's address space (cudaHostAlloc, or
// cudaHostRegister with mapping).  On a GB300 these writes travel over the
// NVLink-C2C host link while the kernel runs, so no copy follows.  Null for
// pageable memory.
void* host_alias(void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

amr_status render_impl(amr_ctx* ctx, int32_t n, const amr_camera* cams, void* const* maps, int32_t* const* counts,
                       int out_on_device, void* cuda_stream, bool partial = false) {
  if (!ctx) return fail(AMR_E_INVALID, "null context");
  if (n < 0 || (n > 0 && (!cams || !maps))) return fail(AMR_E_INVALID, "bad batch arguments");
  if (n == 0) return AMR_OK;
  CUDA_TRY(cudaSetDevice(ctx->device));
  const amr_options opt = ctx->opt;
  std::vector<CamDev> dev(n);
  std::vector<int> precs(n);
  for (int i = 0; i < n; ++i) {
    amr_status st = canonicalise(ctx, cams[i], opt.tile_w, opt.tile_h, dev[i]);
    if (st == AMR_OK) st = attach_pack(ctx, cams[i], dev[i]);
    if (st != AMR_OK) return fail(st, "camera %d: %s", i, g_err.c_str());
    if (!maps[i]) return fail(AMR_E_INVALID, "camera %d: null map pointer", i);
    precs[i] = cams[i].precision;
  }
  cudaStream_t stream = (cudaStream_t)cuda_stream;  // NULL: the CUDA default stream
  if (out_on_device) {
    for (int i = 0; i < n; ++i) {
      dev[i].map = maps[i];
      dev[i].counts = counts ? counts[i] : nullptr;
    }
    LaunchSlot* s = nullptr;
    return enqueue(ctx, opt, dev, precs, stream, &s, partial);
  }
  // Host outputs: a camera whose map (and counts) the GPU can address is
  // written in place; the others go to device staging and are copied back.
  std::vector<char> staged(n, 0);
  std::vector<int64_t> off(n, 0);
  int64_t stage_bytes = 0;
  for (int i = 0; i < n; ++i) {
    void* m = host_alias(maps[i]);
    void* c = (counts && counts[i]) ? host_alias(counts[i]) : nullptr;
    if (m && (c || !(counts && counts[i]))) {
      dev[i].map = m;
      dev[i].counts = (int32_t*)c;
      continue;
    }
    staged[i] = 1;
    off[i] = stage_bytes;
    const int64_t px = (int64_t)cams[i].nx * cams[i].ny;
    stage_bytes += ((map_bytes(cams[i]) + 255) / 256) * 256;
    if (counts && counts[i]) stage_bytes += ((px * 4 + 255) / 256) * 256;
  }
  if (stage_bytes) {
    amr_status st = ensure_stage(ctx, stage_bytes);
    if (st != AMR_OK) return st;
  }
  for (int i = 0; i < n; ++i) {
    if (!staged[i]) continue;
    char* base = (char*)ctx->stage + off[i];
    dev[i].map = base;
    dev[i].counts = (counts && counts[i]) ? (int32_t*)(base + ((map_bytes(cams[i]) + 255) / 256) * 256) : nullptr;
  }
  LaunchSlot* s = nullptr;
  amr_status st = enqueue(ctx, opt, dev, precs, stream, &s);
  if (st != AMR_OK) return st;
  for (int i = 0; i < n; ++i) {
    if (!staged[i]) continue;
    CUDA_TRY(cudaMemcpyAsync(maps[i], dev[i].map, (size_t)map_bytes(cams[i]), cudaMemcpyDeviceToHost, stream));
    if (dev[i].counts)
      CUDA_TRY(cudaMemcpyAsync(counts[i], dev[i].counts, (size_t)cams[i].nx * cams[i].ny * 4, cudaMemcpyDeviceToHost,
                               stream));
  }
  CUDA_TRY(cudaStreamSynchronize(stream));
  return finish_sync(ctx, s);
}

// ------------------------------------------------------------------ server
// Rays per server launch.  A launch renders at most this many rays (whole
// tiles) taken from the admitted requests, so a request that arrives while
// others render joins the next launch (about a millisecond away) instead of
// waiting behind whole batches: continuous batching at tile granularity.
constexpr int64_t kServerLaunchRays = int64_t(1) << 20;

// Deliver a finished request (srv_mu held): status, latency records, its
// budget and arena space back.
void finish_locked(amr_ctx* ctx, const std::shared_ptr<Request>& r, amr_status st, const std::string& err) {
  const auto now = std::chrono::steady_clock::now();
  r->status = st;
  if (!err.empty()) r->err = err;
  r->state = 2;
  r->t_done = now;
  ctx->srv_used -= r->bytes;
  if (r->stage_off >= 0) {
    ctx->arena.give(r->stage_off, r->bytes);
    r->stage_off = -1;
  }
  if (st == AMR_OK) {
    ctx->srv_done++;
    ctx->latencies_ms.push_back(std::chrono::duration<double, std::milli>(now - r->t_submit).count());
    ctx->waits_ms.push_back(std::chrono::duration<double, std::milli>(r->t_start - r->t_submit).count());
    ctx->services_ms.push_back(std::chrono::duration<double, std::milli>(now - r->t_start).count());
  } else {
    ctx->srv_failed++;
  }
  ctx->srv_tlast = now;
}

// Admit queued requests in arrival order while the map-memory budget allows
// (srv_mu held).  A request whose host buffers the GPU can write (page-locked
// and mapped) is rendered straight into them; the others get staging in the
// server's device arena and a copy when their last tile lands.
void admit_locked(amr_ctx* ctx) {
  while (!ctx->queue.empty()) {
    std::shared_ptr<Request> r = ctx->queue.front();
    if (ctx->srv_used + r->bytes > ctx->srv_budget && ctx->srv_used > 0) return;
    CamDev d;
    amr_status cst = canonicalise(ctx, r->cam, ctx->srv_opt.tile_w, ctx->srv_opt.tile_h, d);
    if (cst == AMR_OK) cst = attach_pack(ctx, r->cam, d);
    if (cst != AMR_OK) {
      ctx->queue.pop_front();
      ctx->srv_used += r->bytes;
      finish_locked(ctx, r, cst, g_err);
      ctx->done_cv.notify_all();
      continue;
    }
    void* m = host_alias(r->map);
    void* c = r->counts ? host_alias(r->counts) : nullptr;
    if (m && (c || !r->counts)) {
      d.map = m;
      d.counts = static_cast<int32_t*>(c);
    } else {
      const int64_t off = ctx->arena.take(r->bytes);
      if (off < 0) return;  // fragmented: wait for space
      r->stage_off = off;
      d.map = ctx->arena.base + off;
      d.counts = r->counts ? reinterpret_cast<int32_t*>(ctx->arena.base + off + (map_bytes(r->cam) + 255) / 256 * 256)
                           : nullptr;
    }
    d.tile0 = 0;
    r->dev = d;
    r->tiles = tiles_of(d, ctx->srv_opt.tile_w, ctx->srv_opt.tile_h);
    r->state = 1;
    ctx->srv_used += r->bytes;
    ctx->queue.pop_front();
    ctx->active.push_back(r);
  }
}

void server_worker(amr_ctx* ctx, ServerSlot* slot) {
  cudaSetDevice(ctx->device);
  const int64_t tile_px = (int64_t)ctx->srv_opt.tile_w * ctx->srv_opt.tile_h;
  for (;;) {
    std::vector<std::shared_ptr<Request>> pr;  // the launch's pieces: request, first tile, tiles
    std::vector<int64_t> p0, pk;
    {
      std::unique_lock<std::mutex> lk(ctx->srv_mu);
      ctx->srv_cv.wait(lk, [&] {
        if (ctx->srv_stop) return true;
        admit_locked(ctx);
        for (auto& r : ctx->active)
          if (r->next < r->tiles) return true;
        return false;
      });
      if (ctx->srv_stop) return;
      // Shortest remaining work first: the requests with the fewest tiles not
      // yet handed out go into the launch first, so small requests overtake
      // large ones; at most kServerLaunchRays rays and srv_max_batch requests.
      std::vector<std::shared_ptr<Request>> cand;
      for (auto& r : ctx->active)
        if (r->next < r->tiles) cand.push_back(r);
      std::stable_sort(cand.begin(), cand.end(), [](const std::shared_ptr<Request>& a, const std::shared_ptr<Request>& b) {
        return a->tiles - a->next < b->tiles - b->next;
      });
      int64_t budget = std::max<int64_t>(1, kServerLaunchRays / tile_px);
      const auto now = std::chrono::steady_clock::now();
      for (auto& r : cand) {
        if (budget <= 0 || (int)pr.size() >= ctx->srv_max_batch) break;
        const int64_t k = std::min(r->tiles - r->next, budget);
        if (r->next == 0) r->t_start = now;
        pr.push_back(r);
        p0.push_back(r->next);
        pk.push_back(k);
        r->next += k;
        budget -= k;
      }
      ctx->srv_batches++;
      ctx->srv_inflight++;
      ctx->srv_max_inflight = std::max(ctx->srv_max_inflight, ctx->srv_inflight);
    }
    // One launch over the pieces on this slot's stream.
    std::vector<CamDev> cams(pr.size());
    std::vector<int> precs(pr.size());
    for (size_t i = 0; i < pr.size(); ++i) {
      cams[i] = pr[i]->dev;
      cams[i].tile0 = (int32_t)p0[i];
      precs[i] = pr[i]->cam.precision;
    }
    LaunchSlot* ls = nullptr;
    amr_status st = enqueue(ctx, ctx->srv_opt, cams, precs, slot->stream, &ls, false, &pk);
    std::string err = st == AMR_OK ? std::string() : g_err;
    if (st == AMR_OK) {
      const cudaError_t e = cudaStreamSynchronize(slot->stream);
      if (e != cudaSuccess) {
        st = AMR_E_CUDA;
        err = cudaGetErrorString(e);
      } else if ((st = finish_sync(ctx, ls)) != AMR_OK) {
        err = g_err;
      }
    }
    // Progress; a request whose last tile landed is delivered.
    std::vector<std::shared_ptr<Request>> done;
    {
      std::lock_guard<std::mutex> lk(ctx->srv_mu);
      for (size_t i = 0; i < pr.size(); ++i) {
        auto& r = pr[i];
        if (st != AMR_OK && !r->failed) {
          r->failed = true;
          r->err = err;
        }
        r->finished += pk[i];
        if (r->finished == r->tiles) {
          done.push_back(r);
          ctx->active.erase(std::find(ctx->active.begin(), ctx->active.end(), r));
        }
      }
      ctx->srv_inflight--;
    }
    std::vector<amr_status> out(done.size(), AMR_OK);
    for (size_t i = 0; i < done.size(); ++i) {
      auto& r = done[i];
      if (r->failed) {
        out[i] = AMR_E_CUDA;
        continue;
      }
      if (r->stage_off < 0) continue;
      if (cudaMemcpyAsync(r->map, r->dev.map, (size_t)map_bytes(r->cam), cudaMemcpyDeviceToHost, slot->stream) !=
              cudaSuccess ||
          (r->counts && cudaMemcpyAsync(r->counts, r->dev.counts, (size_t)r->cam.nx * r->cam.ny * 4,
                                        cudaMemcpyDeviceToHost, slot->stream) != cudaSuccess))
        out[i] = AMR_E_CUDA;
    }
    if (!done.empty() && cudaStreamSynchronize(slot->stream) != cudaSuccess)
      for (auto& o : out) o = AMR_E_CUDA;
    {
      std::lock_guard<std::mutex> lk(ctx->srv_mu);
      for (size_t i = 0; i < done.size(); ++i)
        finish_locked(ctx, done[i], out[i], out[i] == AMR_OK ? std::string() : (done[i]->err.empty() ? "CUDA error" : done[i]->err));
    }
    ctx->done_cv.notify_all();
    ctx->srv_cv.notify_all();
  }
}

amr_status start_server(amr_ctx* ctx) {
  if (ctx->srv_started) return AMR_OK;
  ctx->srv_opt = ctx->opt;
  if (cudaMalloc((void**)&ctx->arena.base, (size_t)ctx->srv_budget) != cudaSuccess) {
    cudaGetLastError();
    ctx->arena.base = nullptr;
    return fail(AMR_E_OOM, "cannot allocate the server's %lld-byte map arena", (long long)ctx->srv_budget);
  }
  ctx->arena.reset(ctx->srv_budget);
  for (int i = 0; i < ctx->srv_slots; ++i) {
    auto s = std::make_unique<ServerSlot>();
    CUDA_TRY(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    ctx->srv.push_back(std::move(s));
  }
  for (auto& s : ctx->srv) s->th = std::thread(server_worker, ctx, s.get());
  ctx->srv_started = true;
  ctx->srv_t0 = std::chrono::steady_clock::now();
  return AMR_OK;
}

// Breadth-first renumbering with validation.  order[new] = old oct index.
amr_status linearise(int64_t n, const uint8_t* level, const int32_t* coord, const int32_t* child,
                     std::vector<int32_t>& order, std::vector<uint2>& rec, int& depth) {
  if (level[0] != 1 || coord[0] != 0 || coord[1] != 0 || coord[2] != 0)
    return fail(AMR_E_BADTREE, "oct 0 must be the root: level 1, coord (0,0,0)");
  std::vector<int32_t> seen((size_t)n, -1);
  order.clear();
  order.reserve((size_t)n);
  order.push_back(0);
  seen[0] = 0;
  depth = 1;
  for (size_t p = 0; p < order.size(); ++p) {
    const int64_t o = order[p];
    const int lv = level[o];
    if (lv < 1 || lv > amr::kMaxLevel) return fail(AMR_E_BADTREE, "oct %lld: level %d out of [1, 22]", (long long)o, lv);
    depth = std::max(depth, lv);
    const int64_t lim = int64_t(1) << lv;
    for (int a = 0; a < 3; ++a) {
      const int64_t k = coord[3 * o + a];
      if (k < 0 || k + 1 >= lim + 1 || (k & 1))
        return fail(AMR_E_BADTREE, "oct %lld: coordinate %lld out of range or odd at level %d", (long long)o,
                    (long long)k, lv);
    }
    for (int c = 0; c < 8; ++c) {
      const int64_t ch = child[8 * o + c];
      if (ch == -1) continue;
      if (ch <= 0 || ch >= n) return fail(AMR_E_BADTREE, "oct %lld cell %d: child index %lld out of range", (long long)o, c, (long long)ch);
      if (seen[ch] != -1) return fail(AMR_E_BADTREE, "oct %lld: referenced more than once (cycle or shared child)", (long long)ch);
      if (level[ch] != lv + 1)
        return fail(AMR_E_BADTREE, "oct %lld: level %d but its parent oct %lld has level %d", (long long)ch, level[ch], (long long)o, lv);
      for (int a = 0; a < 3; ++a)
        if (coord[3 * ch + a] != 2 * (coord[3 * o + a] + ((c >> a) & 1)))
          return fail(AMR_E_BADTREE, "oct %lld: coordinates do not match cell %d of parent oct %lld", (long long)ch, c, (long long)o);
      seen[ch] = (int32_t)order.size();
      order.push_back((int32_t)ch);
    }
  }
  if ((int64_t)order.size() != n) {
    for (int64_t o = 0; o < n; ++o)
      if (seen[o] == -1) return fail(AMR_E_BADTREE, "oct %lld: not reachable from the root", (long long)o);
  }
  rec.assign((size_t)n, uint2{0u, 0u});
  for (int64_t p = 0; p < n; ++p) {
    const int64_t o = order[p];
    uint32_t mask = 0, base = 0;
    bool have = false;
    for (int c = 0; c < 8; ++c) {
      const int32_t ch = child[8 * o + c];
      if (ch < 0) continue;
      mask |= 1u << c;
      if (!have) { base = (uint32_t)seen[ch]; have = true; }
    }
    rec[p] = uint2{base, mask | ((uint32_t)level[o] << 8)};
  }
  return AMR_OK;
}

// Face-neighbour links (RAMSES keeps neighbour references per cell, Sec. 1), built in
// breadth-first order from the parent's links.  For oct p and face f = 2 axis +
// (side > 0): the oct of the same level across that face (>= 0), -1 outside
// the box, or -(2 + 8 oct + cell) for the deepest existing cell covering the
// neighbouring region when no oct of p's level exists there (that cell is a
// leaf).
void build_neighbours(const std::vector<uint2>& rec, std::vector<int32_t>& nb) {
  const int64_t n = (int64_t)rec.size();
  nb.assign((size_t)n * 6, -1);
  std::vector<int32_t> parent((size_t)n, -1);
  std::vector<uint8_t> pcell((size_t)n, 0);
  for (int64_t p = 0; p < n; ++p) {
    const uint32_t mask = rec[p].y & 0xffu;
    uint32_t k = rec[p].x;
    for (int c = 0; c < 8; ++c)
      if ((mask >> c) & 1u) {
        parent[k] = (int32_t)p;
        pcell[k] = (uint8_t)c;
        ++k;
      }
  }
  auto child_of = [&](int64_t q, int qc) -> int32_t {
    const uint32_t mask = rec[q].y & 0xffu;
    return (int32_t)(rec[q].x + __builtin_popcount(mask & ((1u << qc) - 1u)));
  };
  for (int64_t p = 1; p < n; ++p) {
    const int64_t par = parent[p];
    const int pc = pcell[p];
    for (int x = 0; x < 3; ++x)
      for (int side = 0; side < 2; ++side) {
        const int f = 2 * x + side;
        const int bit = (pc >> x) & 1;
        int64_t q;
        if (bit != side) {
          q = par;  // the neighbouring region lies inside the parent oct
        } else {
          const int32_t w = nb[(size_t)par * 6 + f];
          if (w < 0) {  // outside, or one coarser leaf covers the parent's neighbour too
            nb[(size_t)p * 6 + f] = w;
            continue;
          }
          q = w;
        }
        const int qc = pc ^ (1 << x);
        if ((rec[q].y >> qc) & 1u) nb[(size_t)p * 6 + f] = child_of(q, qc);
        else nb[(size_t)p * 6 + f] = -(int32_t)(2 + 8 * q + qc);
      }
  }
}

void free_tree(DeviceTree& t) {
  for (const PackedFields& p : t.packs)
    if (p.buf) cudaFree(p.buf);
  if (t.rec) cudaFree(t.rec);
  if (t.nbr) cudaFree(t.nbr);
  for (void* f : t.fields) if (f) cudaFree(f);
  t = DeviceTree{};
}

}  // namespace

namespace amr {

amr_status canonicalise_view(const TreeView& t, const amr_camera& c, int tile_w, CamDev& d) {
  return canonicalise_tree(t, c, tile_w, d);
}

amr_status set_error(amr_status st, const char* msg) { return fail(st, "%s", msg); }

}  // namespace amr

extern "C" {

amr_status amr_create(amr_ctx** out, int device) {
  if (!out) return fail(AMR_E_INVALID, "null output pointer");
  *out = nullptr;
  int ndev = 0;
  CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(AMR_E_INVALID, "device %d of %d", device, ndev);
  CUDA_TRY(cudaSetDevice(device));
  amr_ctx* ctx = new (std::nothrow) amr_ctx;
  if (!ctx) return fail(AMR_E_OOM, "host allocation failed");
  ctx->device = device;
  cudaDeviceProp prop{};
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess ||
      cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete ctx;
    return fail(AMR_E_CUDA, "device set-up failed: %s", cudaGetErrorString(cudaGetLastError()));
  }
  ctx->sms = prop.multiProcessorCount;
  amr_status st = init_slots(ctx);
  if (st != AMR_OK) {
    amr_destroy(ctx);
    return st;
  }
  *out = ctx;
  return AMR_OK;
}

amr_status amr_destroy(amr_ctx* ctx) {
  if (!ctx) return AMR_OK;
  cudaSetDevice(ctx->device);
  {
    std::lock_guard<std::mutex> lk(ctx->srv_mu);
    ctx->srv_stop = true;
    for (auto& r : ctx->queue) {
      r->status = AMR_E_CANCELLED;
      r->state = 2;
    }
    ctx->queue.clear();
  }
  ctx->srv_cv.notify_all();
  ctx->done_cv.notify_all();
  for (auto& s : ctx->srv) {
    if (s->th.joinable()) s->th.join();
    if (s->stream) cudaStreamDestroy(s->stream);
  }
  ctx->srv.clear();
  {
    // Admitted requests whose tiles were not all rendered end cancelled.
    std::lock_guard<std::mutex> lk(ctx->srv_mu);
    for (auto& r : ctx->active) {
      r->status = AMR_E_CANCELLED;
      r->state = 2;
    }
    ctx->active.clear();
  }
  ctx->done_cv.notify_all();
  if (ctx->arena.base) cudaFree(ctx->arena.base);
  cudaDeviceSynchronize();
  for (auto& s : ctx->slots) {
    if (s.start) cudaEventDestroy(s.start);
    if (s.done) cudaEventDestroy(s.done);
    free_slot(s);
  }
  free_tree(ctx->tree);
  if (ctx->stage) cudaFree(ctx->stage);
  if (ctx->blur_tmp) cudaFree(ctx->blur_tmp);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return AMR_OK;
}

amr_status amr_load_octree(amr_ctx* ctx, int64_t n_oct, const uint8_t* level, const int32_t* coord,
                           const int32_t* child, int32_t n_fields, const void* const* fields, int32_t field_dtype) {
  if (!ctx) return fail(AMR_E_INVALID, "null context");
  if (n_oct < 1 || n_oct > (int64_t)0x7fffffff / 8) return fail(AMR_E_INVALID, "n_oct %lld out of range", (long long)n_oct);
  if (!level || !coord || !child) return fail(AMR_E_INVALID, "null tree array");
  if (n_fields < 1 || n_fields > 64 || !fields) return fail(AMR_E_INVALID, "n_fields %d: need 1..64 fields", n_fields);
  for (int f = 0; f < n_fields; ++f)
    if (!fields[f]) return fail(AMR_E_INVALID, "field %d is null", f);
  if (field_dtype != AMR_F32 && field_dtype != AMR_F64) return fail(AMR_E_INVALID, "field dtype %d", field_dtype);
  CUDA_TRY(cudaSetDevice(ctx->device));
  std::vector<int32_t> order;
  std::vector<uint2> rec;
  int depth = 1;
  amr_status st;
  try {
    st = linearise(n_oct, level, coord, child, order, rec, depth);
  } catch (const std::bad_alloc&) {
    return fail(AMR_E_OOM, "host memory for linearisation");
  }
  if (st != AMR_OK) return st;
  std::vector<int32_t> nb;
  try {
    build_neighbours(rec, nb);
    // One 64-byte block per oct: its six links as 8-byte words {link, the
    // linked oct's refinement mask | level << 8} (0 beside -1), then its corner
    // coordinates (even, < 2^22) halved and packed into 64 bits, then the
    // corner marker (the slot a step on several axes reads).
    std::vector<int32_t> blocks((size_t)n_oct * 16, 0);
    for (int64_t p = 0; p < n_oct; ++p) {
      for (int q = 0; q < 6; ++q) {
        const int32_t v = nb[(size_t)p * 6 + q];
        blocks[(size_t)p * 16 + 2 * q] = v;
        uint32_t ry = 0;
        if (v >= 0) ry = rec[v].y;
        else if (v <= -2) ry = rec[(uint32_t)(-v - 2) >> 3].y;
        blocks[(size_t)p * 16 + 2 * q + 1] = (int32_t)ry;
      }
      const int32_t* cc = coord + (size_t)order[p] * 3;
      const uint64_t pk = (uint64_t)(cc[0] >> 1) | ((uint64_t)(cc[1] >> 1) << 21) | ((uint64_t)(cc[2] >> 1) << 42);
      std::memcpy(&blocks[(size_t)p * 16 + 12], &pk, sizeof pk);
      blocks[(size_t)p * 16 + 14] = amr::kCornerLink;
    }
    nb.swap(blocks);
  } catch (const std::bad_alloc&) {
    return fail(AMR_E_OOM, "host memory for neighbour links");
  }
  CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  {
    std::lock_guard<std::mutex> lk(ctx->launch_mu);
    for (auto& s : ctx->slots)
      if (s.pending) {
        cudaEventSynchronize(s.done);
        harvest(ctx, s);
      }
  }
  free_tree(ctx->tree);
  DeviceTree t;
  const size_t esz = field_dtype == AMR_F64 ? 8 : 4;
  const size_t fbytes = (size_t)n_oct * 8 * esz;
  if (cudaMalloc((void**)&t.rec, (size_t)n_oct * sizeof(uint2)) != cudaSuccess) {
    cudaGetLastError();
    return fail(AMR_E_OOM, "device memory for %lld oct records", (long long)n_oct);
  }
  t.fields.assign(n_fields, nullptr);
  for (int f = 0; f < n_fields; ++f) {
    if (cudaMalloc(&t.fields[f], fbytes) != cudaSuccess) {
      cudaGetLastError();
      free_tree(t);
      return fail(AMR_E_OOM, "device memory for field %d (%zu bytes)", f, fbytes);
    }
  }
  if (cudaMalloc((void**)&t.nbr, (size_t)n_oct * 16 * sizeof(int32_t)) != cudaSuccess) {
    cudaGetLastError();
    free_tree(t);
    return fail(AMR_E_OOM, "device memory for %lld neighbour link blocks", (long long)n_oct);
  }
  cudaError_t e = cudaMemcpy(t.rec, rec.data(), (size_t)n_oct * sizeof(uint2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(t.nbr, nb.data(), (size_t)n_oct * 16 * sizeof(int32_t), cudaMemcpyHostToDevice);
  std::vector<char> buf;
  try {
    buf.resize(fbytes);
  } catch (const std::bad_alloc&) {
    free_tree(t);
    return fail(AMR_E_OOM, "host memory for field permutation");
  }
  for (int f = 0; f < n_fields && e == cudaSuccess; ++f) {
    const char* src = (const char*)fields[f];
    for (int64_t p = 0; p < n_oct; ++p) std::memcpy(&buf[(size_t)p * 8 * esz], src + (size_t)order[p] * 8 * esz, 8 * esz);
    e = cudaMemcpy(t.fields[f], buf.data(), fbytes, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    free_tree(t);
    return fail(AMR_E_CUDA, "tree upload: %s", cudaGetErrorString(e));
  }
  t.n_oct = n_oct;
  t.depth = depth;
  t.f64 = field_dtype == AMR_F64;
  t.bytes = (int64_t)(n_oct * (sizeof(uint2) + 16 * sizeof(int32_t)) + n_fields * fbytes);
  ctx->tree = std::move(t);
  return AMR_OK;
}

amr_status amr_render(amr_ctx* ctx, const amr_camera* cam, void* map_out, int32_t* count_out, int out_on_device,
                      void* cuda_stream) {
  if (!cam || !map_out) return fail(AMR_E_INVALID, "null camera or map");
  void* maps[1] = {map_out};
  int32_t* counts[1] = {count_out};
  return render_impl(ctx, 1, cam, maps, counts, out_on_device, cuda_stream);
}

amr_status amr_render_batch(amr_ctx* ctx, int32_t n, const amr_camera* cams, void* const* maps,
                            int32_t* const* counts, int out_on_device, void* cuda_stream) {
  return render_impl(ctx, n, cams, maps, counts, out_on_device, cuda_stream);
}

amr_status amr_render_batch_partial(amr_ctx* ctx, int32_t n, const amr_camera* cams, void* const* partials,
                                    int32_t* const* counts, void* cuda_stream) {
  return render_impl(ctx, n, cams, partials, counts, 1, cuda_stream, true);
}

amr_status amr_slice(amr_ctx* ctx, const amr_camera* cam, void* map_out, int32_t* level_out, int out_on_device,
                     void* cuda_stream) {
  if (!ctx || !cam || !map_out) return fail(AMR_E_INVALID, "null argument");
  CUDA_TRY(cudaSetDevice(ctx->device));
  amr_camera c = *cam;
  c.mode = AMR_MODE_COLUMN;  // the slice reads field_value only
  CamDev d;
  amr_status st = canonicalise(ctx, c, ctx->opt.tile_w, ctx->opt.tile_h, d);
  if (st != AMR_OK) return st;
  const bool out64 = cam->precision == AMR_PREC_FP64;
  const int64_t px = (int64_t)c.nx * c.ny;
  const int64_t mbytes = px * (out64 ? 8 : 4);
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  LaunchSlot* s = nullptr;
  if (out_on_device) {
    d.map = map_out;
    d.counts = level_out;
    return enqueue_slice(ctx, d, out64, stream, &s);
  }
  // Page-locked host outputs the GPU can address are written in place.
  void* hm = host_alias(map_out);
  void* hl = level_out ? host_alias(level_out) : nullptr;
  if (hm && (hl || !level_out)) {
    d.map = hm;
    d.counts = (int32_t*)hl;
    st = enqueue_slice(ctx, d, out64, stream, &s);
    if (st != AMR_OK) return st;
    CUDA_TRY(cudaStreamSynchronize(stream));
    return finish_sync(ctx, s);
  }
  const int64_t moff = ((mbytes + 255) / 256) * 256;
  st = ensure_stage(ctx, moff + (level_out ? px * 4 : 0));
  if (st != AMR_OK) return st;
  d.map = ctx->stage;
  d.counts = level_out ? (int32_t*)((char*)ctx->stage + moff) : nullptr;
  st = enqueue_slice(ctx, d, out64, stream, &s);
  if (st != AMR_OK) return st;
  CUDA_TRY(cudaMemcpyAsync(map_out, d.map, (size_t)mbytes, cudaMemcpyDeviceToHost, stream));
  if (level_out) CUDA_TRY(cudaMemcpyAsync(level_out, d.counts, (size_t)px * 4, cudaMemcpyDeviceToHost, stream));
  CUDA_TRY(cudaStreamSynchronize(stream));
  return finish_sync(ctx, s);
}

amr_status amr_blur(amr_ctx* ctx, int32_t nx, int32_t ny, const float* in, const float* level, double pixel,
                    float* out, void* cuda_stream) {
  if (!ctx || !in || !level || !out) return fail(AMR_E_INVALID, "null argument");
  if (nx <= 0 || ny <= 0 || (int64_t)nx * ny >= (int64_t(1) << 31)) return fail(AMR_E_INVALID, "map size %d x %d", nx, ny);
  if (!(pixel > 0.0) || !std::isfinite(pixel)) return fail(AMR_E_INVALID, "pixel size must be positive");
  if (in == out) return fail(AMR_E_INVALID, "in and out alias");
  CUDA_TRY(cudaSetDevice(ctx->device));
  const int64_t bytes = (int64_t)nx * ny * 4;
  if (ctx->blur_cap < bytes) {
    if (ctx->blur_tmp) {
      CUDA_TRY(cudaDeviceSynchronize());
      cudaFree(ctx->blur_tmp);
    }
    ctx->blur_tmp = nullptr;
    ctx->blur_cap = 0;
    if (cudaMalloc(&ctx->blur_tmp, (size_t)bytes) != cudaSuccess) {
      cudaGetLastError();
      return fail(AMR_E_OOM, "blur buffer of %lld bytes", (long long)bytes);
    }
    ctx->blur_cap = bytes;
  }
  CUDA_TRY(amr::launch_blur(in, level, pixel, (float*)ctx->blur_tmp, out, nx, ny, (cudaStream_t)cuda_stream));
  return AMR_OK;
}

amr_status amr_camera_check(amr_ctx* ctx, const amr_camera* cam, int32_t* level_out) {
  if (!ctx || !cam) return fail(AMR_E_INVALID, "null argument");
  CamDev d;
  amr_status st = canonicalise(ctx, *cam, ctx->opt.tile_w, ctx->opt.tile_h, d);
  if (st == AMR_OK && level_out) *level_out = d.L;
  return st;
}

amr_status amr_set_options(amr_ctx* ctx, const amr_options* opt) {
  if (!ctx || !opt) return fail(AMR_E_INVALID, "null argument");
  amr_status st = check_options(*opt);
  if (st != AMR_OK) return st;
  ctx->opt = *opt;
  return AMR_OK;
}

amr_status amr_get_options(amr_ctx* ctx, amr_options* opt) {
  if (!ctx || !opt) return fail(AMR_E_INVALID, "null argument");
  *opt = ctx->opt;
  return AMR_OK;
}

amr_status amr_autotune(amr_ctx* ctx, int32_t n, const amr_camera* cams, int32_t reps, amr_options* best,
                        double* ms_out) {
  if (!ctx || n <= 0 || !cams || reps < 1) return fail(AMR_E_INVALID, "bad autotune arguments");
  CUDA_TRY(cudaSetDevice(ctx->device));
  // Device outputs into staging; every candidate renders the same batch.
  int64_t bytes = 0;
  for (int i = 0; i < n; ++i) bytes += ((map_bytes(cams[i]) + 255) / 256) * 256;
  amr_status st = ensure_stage(ctx, bytes);
  if (st != AMR_OK) return st;
  std::vector<void*> maps(n);
  int64_t off = 0;
  for (int i = 0; i < n; ++i) {
    maps[i] = (char*)ctx->stage + off;
    off += ((map_bytes(cams[i]) + 255) / 256) * 256;
  }
  const int tiles[][2] = {{8, 4}, {4, 8}, {16, 2}, {32, 1}};
  const int blocks[] = {128, 256};
  const int grabs[] = {1, 4};
  const amr_options saved = ctx->opt;
  amr_options bestopt = saved;
  double bestms = 1e300;
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  // Median of `reps` timed runs of one candidate (a first run warms caches).
  auto try_opt = [&](const amr_options& o) {
    ctx->opt = o;
    std::vector<double> times;
    for (int r = 0; r < reps + 1 && st == AMR_OK; ++r) {
      cudaEventRecord(e0, ctx->stream);
      st = render_impl(ctx, n, cams, maps.data(), nullptr, 1, ctx->stream);
      cudaEventRecord(e1, ctx->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) st = fail(AMR_E_CUDA, "autotune sync failed");
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0) times.push_back(ms);
    }
    if (st != AMR_OK) return;
    std::sort(times.begin(), times.end());
    const double med = times[times.size() / 2];
    if (med < bestms) {
      bestms = med;
      bestopt = o;
    }
  };
  // First the launch shapes at the context's register cap, then the other
  // caps at the best shape.
  for (auto& tl : tiles)
    for (int bt : blocks)
      for (int gr : grabs) {
        if (st != AMR_OK) break;
        amr_options o = saved;
        o.tile_w = tl[0];
        o.tile_h = tl[1];
        o.block_threads = bt;
        o.tiles_per_grab = gr;
        o.blocks_per_sm = 0;
        try_opt(o);
      }
  const int shape_regs = saved.max_regs ? saved.max_regs : amr::kDefaultRegs;
  const amr_options best_shape = bestopt;
  for (int regs : amr::kRegCaps) {
    if (st != AMR_OK || regs == shape_regs) continue;
    amr_options o = best_shape;
    o.max_regs = regs;
    try_opt(o);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->opt = st == AMR_OK ? bestopt : saved;
  if (st != AMR_OK) return st;
  {
    std::lock_guard<std::mutex> lk(ctx->launch_mu);
    for (auto& s : ctx->slots)
      if (s.pending) {
        cudaEventSynchronize(s.done);
        harvest(ctx, s);
      }
  }
  ctx->autotune_ms = bestms;
  if (best) *best = bestopt;
  if (ms_out) *ms_out = bestms;
  return AMR_OK;
}

amr_status amr_server_config(amr_ctx* ctx, int32_t slots, int64_t map_budget_bytes, int32_t max_batch) {
  if (!ctx) return fail(AMR_E_INVALID, "null context");
  std::lock_guard<std::mutex> lk(ctx->srv_mu);
  if (ctx->srv_started) return fail(AMR_E_BUSY, "server already running");
  if (slots < 1 || slots > 8 || map_budget_bytes < 0 || max_batch < 1)
    return fail(AMR_E_INVALID, "server config: slots 1..8, budget >= 0, max_batch >= 1");
  ctx->srv_slots = slots;
  ctx->srv_budget = map_budget_bytes ? map_budget_bytes : (int64_t(1) << 30);
  ctx->srv_max_batch = max_batch;
  return AMR_OK;
}

amr_status amr_submit(amr_ctx* ctx, const amr_camera* cam, void* map, int32_t* counts, uint64_t* ticket) {
  if (!ctx || !cam || !map || !ticket) return fail(AMR_E_INVALID, "null argument");
  CamDev d;
  amr_status st = canonicalise(ctx, *cam, ctx->opt.tile_w, ctx->opt.tile_h, d);
  if (st != AMR_OK) return st;
  auto r = std::make_shared<Request>();
  r->cam = *cam;
  r->map = map;
  r->counts = counts;
  r->bytes = ((map_bytes(*cam) + 255) / 256) * 256 + (counts ? (((int64_t)cam->nx * cam->ny * 4 + 255) / 256) * 256 : 0);
  r->t_submit = std::chrono::steady_clock::now();
  std::lock_guard<std::mutex> lk(ctx->srv_mu);
  if (ctx->srv_stop) return fail(AMR_E_CANCELLED, "context is shutting down");
  if ((int)ctx->queue.size() >= ctx->srv_max_queue) return fail(AMR_E_BUSY, "request queue full");
  if (r->bytes > ctx->srv_budget) return fail(AMR_E_OOM, "request needs %lld bytes, budget %lld", (long long)r->bytes, (long long)ctx->srv_budget);
  if (!ctx->srv_started) {
    st = start_server(ctx);
    if (st != AMR_OK) return st;
  }
  *ticket = ctx->next_ticket++;
  ctx->reqs[*ticket] = r;
  ctx->queue.push_back(r);
  ctx->srv_cv.notify_one();
  return AMR_OK;
}

amr_status amr_wait(amr_ctx* ctx, uint64_t ticket, int64_t timeout_us) {
  if (!ctx) return fail(AMR_E_INVALID, "null context");
  std::unique_lock<std::mutex> lk(ctx->srv_mu);
  auto it = ctx->reqs.find(ticket);
  if (it == ctx->reqs.end()) return fail(AMR_E_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
  std::shared_ptr<Request> r = it->second;
  auto pred = [&] { return r->state == 2; };
  if (timeout_us < 0) {
    ctx->done_cv.wait(lk, pred);
  } else if (!ctx->done_cv.wait_for(lk, std::chrono::microseconds(timeout_us), pred)) {
    return fail(AMR_E_TIMEOUT, "ticket %llu not finished after %lld us", (unsigned long long)ticket, (long long)timeout_us);
  }
  ctx->reqs.erase(ticket);
  if (r->status != AMR_OK) return fail(r->status, "request %llu failed: %s", (unsigned long long)ticket, r->err.c_str());
  return AMR_OK;
}

amr_status amr_cancel(amr_ctx* ctx, uint64_t ticket) {
  if (!ctx) return fail(AMR_E_INVALID, "null context");
  std::lock_guard<std::mutex> lk(ctx->srv_mu);
  auto it = ctx->reqs.find(ticket);
  if (it == ctx->reqs.end()) return fail(AMR_E_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
  auto r = it->second;
  if (r->state != 0) return fail(AMR_E_BUSY, "ticket %llu already running or done", (unsigned long long)ticket);
  for (auto q = ctx->queue.begin(); q != ctx->queue.end(); ++q)
    if (q->get() == r.get()) {
      ctx->queue.erase(q);
      break;
    }
  r->status = AMR_E_CANCELLED;
  r->err = "cancelled";
  r->state = 2;
  ctx->done_cv.notify_all();
  return AMR_OK;
}

amr_status amr_stats(amr_ctx* ctx, char* json_buf, int64_t buf_len) {
  if (!ctx || !json_buf || buf_len <= 0) return fail(AMR_E_INVALID, "bad arguments");
  cudaSetDevice(ctx->device);
  {
    std::lock_guard<std::mutex> lk(ctx->launch_mu);
    for (auto& s : ctx->slots)
      if (s.pending && cudaEventQuery(s.done) == cudaSuccess) harvest(ctx, s);
    cudaGetLastError();
  }
  double p50 = 0, p99 = 0, fps = 0, w50 = 0, w99 = 0, s50 = 0, s99 = 0;
  int64_t done, failed, batches, maxin, queued;
  {
    std::lock_guard<std::mutex> lk(ctx->srv_mu);
    auto pct = [](std::vector<double> l, double* a, double* b) {
      if (l.empty()) return;
      std::sort(l.begin(), l.end());
      *a = l[(size_t)(0.50 * (l.size() - 1))];
      *b = l[(size_t)(0.99 * (l.size() - 1))];
    };
    pct(ctx->latencies_ms, &p50, &p99);
    pct(ctx->waits_ms, &w50, &w99);
    pct(ctx->services_ms, &s50, &s99);
    if (!ctx->latencies_ms.empty()) {
      const double span = std::chrono::duration<double>(ctx->srv_tlast - ctx->srv_t0).count();
      fps = span > 0 ? ctx->latencies_ms.size() / span : 0.0;
    }
    done = ctx->srv_done;
    failed = ctx->srv_failed;
    batches = ctx->srv_batches;
    maxin = ctx->srv_max_inflight;
    queued = (int64_t)ctx->queue.size();
  }
  const amr_options& o = ctx->opt;
  const bool f64 = ctx->tree.f64;
  const int regs = o.max_regs ? o.max_regs : amr::kDefaultRegs;
  int64_t packed_bytes = 0;
  int n_packs = 0;
  {
    std::lock_guard<std::mutex> lk(ctx->pack_mu);
    for (const PackedFields& p : ctx->tree.packs) packed_bytes += p.bytes;
    n_packs = (int)ctx->tree.packs.size();
  }
  char buf[2048];
  int len = std::snprintf(
      buf, sizeof buf,
      "{\"renders\": %lld, \"cameras\": %lld, \"rays\": %lld, \"segments\": %llu, \"h2d_bytes\": %lld, \"device_errors\": %lld, "
      "\"last_batch_ms\": %.6f, \"tree\": {\"n_oct\": %lld, \"depth\": %d, \"device_bytes\": %lld, \"f64\": %d, "
      "\"packed_fields\": %d, \"packed_bytes\": %lld}, "
      "\"options\": {\"tile_w\": %d, \"tile_h\": %d, \"block_threads\": %d, \"blocks_per_sm\": %d, "
      "\"tiles_per_grab\": %d, \"use_graph\": %d, \"max_regs\": %d}, \"autotune_ms\": %.6f, \"graph_captures\": %lld, \"graph_launches\": %lld, "
      "\"regs\": {\"fp64\": %d, \"fp32_kahan\": %d, \"fp32_plain\": %d}, \"sms\": %d, "
      "\"server\": {\"done\": %lld, \"failed\": %lld, \"batches\": %lld, \"max_inflight\": %lld, \"queued\": %lld, "
      "\"p50_ms\": %.6f, \"p99_ms\": %.6f, \"wait_p50_ms\": %.6f, \"wait_p99_ms\": %.6f, "
      "\"service_p50_ms\": %.6f, \"service_p99_ms\": %.6f, \"frames_per_s\": %.6f}}",
      (long long)ctx->n_renders, (long long)ctx->n_cams, (long long)ctx->n_rays, ctx->n_segments,
      (long long)ctx->n_h2d_bytes, (long long)ctx->n_dev_errors, ctx->last_batch_ms, (long long)ctx->tree.n_oct, ctx->tree.depth,
      (long long)ctx->tree.bytes, f64 ? 1 : 0, n_packs, (long long)packed_bytes, o.tile_w, o.tile_h, o.block_threads, o.blocks_per_sm, o.tiles_per_grab,
      o.use_graph, o.max_regs, ctx->autotune_ms, (long long)ctx->n_graph_captures, (long long)ctx->n_graph_launches,
      amr::batch_regs(0, f64, true, regs), amr::batch_regs(1, f64, true, regs), amr::batch_regs(2, f64, true, regs),
      ctx->sms, (long long)done, (long long)failed, (long long)batches, (long long)maxin, (long long)queued, p50, p99,
      w50, w99, s50, s99, fps);
  if (len < 0) return fail(AMR_E_INVALID, "stats formatting failed");
  int64_t n = std::min<int64_t>(len, buf_len - 1);
  std::memcpy(json_buf, buf, (size_t)n);
  json_buf[n] = '\0';
  return AMR_OK;
}

amr_status amr_tree_info(amr_ctx* ctx, int64_t* n_oct, int32_t* depth, int64_t* device_bytes) {
  if (!ctx) return fail(AMR_E_INVALID, "null context");
  if (n_oct) *n_oct = ctx->tree.n_oct;
  if (depth) *depth = ctx->tree.depth;
  if (device_bytes) *device_bytes = ctx->tree.bytes;
  return AMR_OK;
}

const char* amr_last_error(amr_ctx* ctx) {
  (void)ctx;
  return g_err.c_str();
}

}  // extern "C"

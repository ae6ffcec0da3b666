// amr_render_batch_noalloc: the batch renderer for callers that cannot
// allocate GPU memory.
//
// Who needs it: a renderer embedded in a running simulation (in-situ
// visualisation), where the simulation's own memory manager owns the GPU and
// forbids other allocations; latency-critical loops, where a cudaMalloc or
// cudaFree could stall on a device-wide synchronisation; processes that must
// keep a fixed, pre-declared memory footprint.  Such callers keep the octree in
// their own device buffers and pass it in with the cameras and output maps.
//
// The batch kernel's scratch (camera table, tile prefix sums, work-queue head,
// error word and segment counter) lives in one file-scope __device__ array of
// fixed size instead of context memory.  Every GPU that loads this library
// holds that array until the process exits.  All calls share it: the queue
// blocks are cleared on every call, and calls whose work overlaps on the GPU
// (different streams, or different host threads with no ordering) race on it.
#include <cstdio>
#include <mutex>

#include "amr.h"
#include "amr_internal.h"

namespace {

constexpr int kMaxCams = AMR_NOALLOC_MAX_CAMERAS;
constexpr size_t kAlign = 256;
constexpr size_t up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kCamBytes = sizeof(amr::CamDev) * kMaxCams;
constexpr size_t kTileInts = (size_t)amr::kMaxPrecisions * (kMaxCams + 1);
constexpr size_t kTilesOff = up(kCamBytes);
constexpr size_t kQueueOff = kTilesOff + up(kTileInts * sizeof(int32_t));
constexpr size_t kScratchBytes = kQueueOff + up(amr::kMaxPrecisions * sizeof(amr::QueueBlock));
static_assert(kScratchBytes <= 224 * 1024, "no-allocation scratch must stay modest");

constexpr int kMaxDevices = 64;

}  // namespace

// The scratch itself.  Host code must not use this name as an address: it only
// stands for the symbol; the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

std::mutex g_mu;                 // serialises set-up and the host staging below
void* g_scratch[kMaxDevices];    // device address of g_noalloc_scratch, per device
int g_sms[kMaxDevices];
bool g_ready[kMaxDevices];
amr::CamDev g_cams[kMaxCams];    // host staging, grouped by precision
int32_t g_tiles[kTileInts];

int32_t failf(int32_t st, const char* fmt, long long a, long long b = 0) {
  char msg[256];
  std::snprintf(msg, sizeof msg, fmt, a, b);
  return amr::set_error(st, msg);
}

// Once per device, with that device current: the scratch's device address and
// the SM count.  The first call on each device does this.
int32_t setup(int dev, unsigned char** scratch, int* sms) {
  if (!g_ready[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return amr::set_error(AMR_E_CUDA, cudaGetErrorString(e));
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return amr::set_error(AMR_E_CUDA, cudaGetErrorString(e));
    g_scratch[dev] = p;
    g_sms[dev] = n;
    g_ready[dev] = true;
  }
  *scratch = static_cast<unsigned char*>(g_scratch[dev]);
  *sms = g_sms[dev];
  return AMR_OK;
}

}  // namespace

extern "C" amr_status amr_render_batch_noalloc(int64_t n_oct, const uint64_t* records, int32_t depth,
                                               int32_t n_fields, const void* const* fields, int32_t field_dtype,
                                               int32_t n, const amr_camera* cams, void* const* maps,
                                               int32_t* const* counts, void* cuda_stream) {
  if (n < 0 || n > kMaxCams)
    return failf(AMR_E_INVALID, "%lld cameras: the no-allocation batch holds at most %lld", n, kMaxCams);
  if (n_oct < 1 || n_oct > (int64_t)0x7fffffff / 8 || !records)
    return failf(AMR_E_INVALID, "n_oct %lld out of range or null records", n_oct);
  if (depth < 1 || depth > amr::kMaxLevel) return failf(AMR_E_INVALID, "tree depth %lld out of [1, 22]", depth);
  if (n_fields < 1 || n_fields > 64 || !fields) return failf(AMR_E_INVALID, "n_fields %lld: need 1..64", n_fields);
  for (int f = 0; f < n_fields; ++f)
    if (!fields[f]) return failf(AMR_E_INVALID, "field %lld is null", f);
  if (field_dtype != AMR_F32 && field_dtype != AMR_F64) return failf(AMR_E_INVALID, "field dtype %lld", field_dtype);
  if (n == 0) return AMR_OK;
  if (!cams || !maps) return amr::set_error(AMR_E_INVALID, "null cameras or maps");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return amr::set_error(AMR_E_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return failf(AMR_E_INVALID, "device %lld beyond %lld", dev, kMaxDevices);

  std::lock_guard<std::mutex> lk(g_mu);
  unsigned char* scratch = nullptr;
  int sms = 0;
  int32_t st = setup(dev, &scratch, &sms);
  if (st != AMR_OK) return st;

  const int tile_w = 8, tile_h = 4, block = 256;
  const amr::TreeView view{fields, n_fields, depth, true};
  // Canonicalise every camera and place it in its precision group.
  int groups[amr::kMaxPrecisions] = {0, 0, 0};
  for (int i = 0; i < n; ++i) {
    if (cams[i].precision < AMR_PREC_FP64 || cams[i].precision > AMR_PREC_FP32_PLAIN)
      return failf(AMR_E_INVALID, "camera %lld: unknown precision %lld", i, cams[i].precision);
    groups[cams[i].precision]++;
  }
  int gstart[amr::kMaxPrecisions + 1] = {0, groups[0], groups[0] + groups[1], n};
  int fill[amr::kMaxPrecisions] = {gstart[0], gstart[1], gstart[2]};
  for (int i = 0; i < n; ++i) {
    if (!maps[i]) return failf(AMR_E_INVALID, "camera %lld: null map", i);
    amr::CamDev& d = g_cams[fill[cams[i].precision]++];
    st = amr::canonicalise_view(view, cams[i], tile_w, d);
    if (st != AMR_OK) return st;
    d.map = maps[i];
    d.counts = counts ? counts[i] : nullptr;
  }
  int64_t total[amr::kMaxPrecisions] = {0, 0, 0};
  for (int g = 0; g < amr::kMaxPrecisions; ++g) {
    int32_t* tp = g_tiles + (size_t)g * (kMaxCams + 1);
    int64_t acc = 0;
    for (int i = 0; i < groups[g]; ++i) {
      const amr::CamDev& d = g_cams[gstart[g] + i];
      tp[i] = (int32_t)acc;
      acc += (int64_t)((d.nx + tile_w - 1) / tile_w) * ((d.ny + tile_h - 1) / tile_h);
    }
    tp[groups[g]] = (int32_t)acc;
    if (acc >= (int64_t(1) << 31) - 4096) return failf(AMR_E_INVALID, "batch too large: %lld tiles", acc);
    total[g] = acc;
  }

  // Upload into the shared scratch (pageable copies: the staging above may be
  // reused once they return), clear the queue blocks, launch per precision.
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  amr::CamDev* d_cams = reinterpret_cast<amr::CamDev*>(scratch);
  int32_t* d_tiles = reinterpret_cast<int32_t*>(scratch + kTilesOff);
  amr::QueueBlock* d_q = reinterpret_cast<amr::QueueBlock*>(scratch + kQueueOff);
  e = cudaMemcpyAsync(d_cams, g_cams, (size_t)n * sizeof(amr::CamDev), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_tiles, g_tiles, kTileInts * sizeof(int32_t), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_q, 0, amr::kMaxPrecisions * sizeof(amr::QueueBlock), stream);
  const bool f64 = field_dtype == AMR_F64;
  for (int g = 0; g < amr::kMaxPrecisions && e == cudaSuccess; ++g) {
    if (!groups[g] || !total[g]) continue;
    amr::BatchArgs a{};
    a.rec = reinterpret_cast<const uint2*>(records);
    a.n_oct = (uint32_t)n_oct;
    a.n_cams = groups[g];
    a.cams = d_cams + gstart[g];
    a.tile_start = d_tiles + (size_t)g * (kMaxCams + 1);
    a.total_tiles = (int32_t)total[g];
    a.tile_w = tile_w;
    a.tile_h = tile_h;
    a.tiles_per_grab = 1;
    a.q = d_q + g;
    int bps = 1;
    e = amr::batch_occupancy(g, f64, false, block, amr::kDefaultRegs, &bps);
    if (e != cudaSuccess) break;
    const int64_t blocks_needed = (total[g] * 32 + block - 1) / block;
    int64_t grid = (int64_t)sms * (bps > 0 ? bps : 1);
    grid = grid < blocks_needed ? grid : blocks_needed;
    e = amr::launch_batch(g, f64, a, (int)(grid > 0 ? grid : 1), block, amr::kDefaultRegs, stream);
  }
  if (e != cudaSuccess) return amr::set_error(AMR_E_CUDA, cudaGetErrorString(e));
  return AMR_OK;
}

// Device status of the last no-allocation batch on the current device: the
// queue blocks' error words and segment counters, read back into the caller's
// host memory after the stream drains.  The copy lands in this function's own
// stack, so nothing is allocated.
extern "C" amr_status amr_noalloc_status(void* cuda_stream, int32_t* host_error, int32_t* host_oct,
                                         uint64_t* host_segments) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return amr::set_error(AMR_E_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return failf(AMR_E_INVALID, "device %lld beyond %lld", dev, kMaxDevices);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ready[dev]) return amr::set_error(AMR_E_INVALID, "no no-allocation batch has run on this device");
  amr::QueueBlock q[amr::kMaxPrecisions];
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  const unsigned char* scratch = static_cast<const unsigned char*>(g_scratch[dev]);
  e = cudaMemcpyAsync(q, scratch + kQueueOff, sizeof q, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return amr::set_error(AMR_E_CUDA, cudaGetErrorString(e));
  int32_t err = amr::kDevOk, oct = -1;
  uint64_t segs = 0;
  for (int g = 0; g < amr::kMaxPrecisions; ++g) {
    segs += q[g].segments;
    if (err == amr::kDevOk && q[g].error != amr::kDevOk) {
      err = q[g].error;
      oct = q[g].err_oct;
    }
  }
  if (host_error) *host_error = err;
  if (host_oct) *host_oct = oct;
  if (host_segments) *host_segments = segs;
  return AMR_OK;
}

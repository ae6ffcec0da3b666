// Sort-last merge of partial renders (Sec. 3.1: the octree is split among
// processes, each renders its own part, and the partial images are combined).
//
// Sec. 2.2 adds the leaves' contributions without any ordering, so a ray's
// sums over disjoint leaf domains add up to its sum over the whole tree, and
// its maximum is the maximum of the domains' maxima.  A partial render (see
// amr_render_batch_partial) stores each pixel's accumulators instead of the
// finished value: FP32 sums as (high, low) pairs whose sum is the value (the
// compensated form the kernel keeps), FP64 sums as plain doubles.  This kernel
// adds the domains' pairs with error-free transformations (Knuth's TwoSum:
// s + t = a + b exactly), carries every rounding error and low part in a
// second accumulator, and only then divides the weighted mean.  One thread per
// pixel; all reads are coalesced and each partial is read once, so the merge
// is bound by HBM bandwidth, provided each thread keeps several reads in
// flight: the FP32 paths issue four domains' loads before adding them.
#include <cuda_runtime.h>

#include <cstdio>

#include "amr.h"
#include "amr_internal.h"

namespace amr {
namespace {

constexpr int kMaxParts = AMR_MERGE_MAX_PARTS;

struct MergeArgs {
  const void* parts[kMaxParts];
  int32_t n_parts;
  int32_t mode;
  int64_t n_px;
  void* out;
};

__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double fadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double fsub(double a, double b) { return __dsub_rn(a, b); }

// Knuth's TwoSum: s = fl(a + b) and the exact error t, s + t = a + b (six
// round-to-nearest operations, no branch, any magnitudes).
template <typename T>
__device__ __forceinline__ T two_sum(T a, T b, T& t) {
  const T s = fadd(a, b);
  const T bv = fsub(s, a);
  t = fadd(fsub(a, fsub(s, bv)), fsub(b, bv));
  return s;
}

// Sum of n (high, low) pairs: high parts through TwoSum, every error and low
// part into e; the value is s + e.
template <typename T>
struct CSum {
  T s = 0, e = 0;
  __device__ __forceinline__ void add(T hi, T lo) {
    T t;
    s = two_sum(s, hi, t);
    e = fadd(e, fadd(t, lo));
  }
  __device__ __forceinline__ T value() const { return fadd(s, e); }
};

template <typename T>
__global__ void __launch_bounds__(256) merge_kernel(const MergeArgs a) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const bool weighted = a.mode == AMR_MODE_WMEAN || a.mode == AMR_MODE_LEVEL;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < a.n_px; p += stride) {
    T v;
    if (a.mode == AMR_MODE_MAX) {
      v = 0;
      for (int d = 0; d < a.n_parts; ++d) v = fmax(v, __ldg(static_cast<const T*>(a.parts[d]) + p));
    } else if (sizeof(T) == 4) {
      // FP32 partials: column (s, c) float2; weighted (S, cS, N, cN) float4.
      // Four domains' loads are issued before their sums, so each thread has
      // four reads in flight (the additions keep the domain order).
      CSum<float> S, N;
      int d = 0;
      if (weighted) {
        for (; d + 4 <= a.n_parts; d += 4) {
          float4 q[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) q[u] = __ldg(static_cast<const float4*>(a.parts[d + u]) + p);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            S.add(q[u].x, q[u].y);
            N.add(q[u].z, q[u].w);
          }
        }
        for (; d < a.n_parts; ++d) {
          const float4 q = __ldg(static_cast<const float4*>(a.parts[d]) + p);
          S.add(q.x, q.y);
          N.add(q.z, q.w);
        }
      } else {
        for (; d + 4 <= a.n_parts; d += 4) {
          float2 q[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) q[u] = __ldg(static_cast<const float2*>(a.parts[d + u]) + p);
#pragma unroll
          for (int u = 0; u < 4; ++u) S.add(q[u].x, q[u].y);
        }
        for (; d < a.n_parts; ++d) {
          const float2 q = __ldg(static_cast<const float2*>(a.parts[d]) + p);
          S.add(q.x, q.y);
        }
      }
      const float s = S.value();
      v = (T)s;
      if (weighted) v = (T)(s != 0.0f ? __fdiv_rn(N.value(), s) : 0.0f);
    } else {
      // FP64 partials: column double; weighted (S, N) double2.
      CSum<double> S, N;
      for (int d = 0; d < a.n_parts; ++d) {
        if (weighted) {
          const double2 q = __ldg(static_cast<const double2*>(a.parts[d]) + p);
          S.add(q.x, 0.0);
          N.add(q.y, 0.0);
        } else {
          S.add(__ldg(static_cast<const double*>(a.parts[d]) + p), 0.0);
        }
      }
      const double s = S.value();
      v = (T)s;
      if (weighted) v = (T)(s != 0.0 ? __ddiv_rn(N.value(), s) : 0.0);
    }
    static_cast<T*>(a.out)[p] = v;
  }
}

}  // namespace
}  // namespace amr

extern "C" amr_status amr_merge_partials(int32_t n_parts, int32_t mode, int32_t precision, int64_t n_px,
                                         const void* const* partials, void* map_out, void* cuda_stream) {
  char msg[160];
  if (n_parts < 1 || n_parts > amr::kMaxParts) {
    std::snprintf(msg, sizeof msg, "%d partials: merge 1..%d", n_parts, amr::kMaxParts);
    return amr::set_error(AMR_E_INVALID, msg);
  }
  if (mode < AMR_MODE_COLUMN || mode > AMR_MODE_LEVEL) return amr::set_error(AMR_E_INVALID, "unknown mode");
  if (precision < AMR_PREC_FP64 || precision > AMR_PREC_FP32_PLAIN)
    return amr::set_error(AMR_E_INVALID, "unknown precision");
  if (n_px < 0 || (n_px > 0 && (!partials || !map_out))) return amr::set_error(AMR_E_INVALID, "bad buffers");
  if (n_px == 0) return AMR_OK;
  amr::MergeArgs a{};
  for (int d = 0; d < n_parts; ++d) {
    if (!partials[d]) return amr::set_error(AMR_E_INVALID, "null partial map");
    a.parts[d] = partials[d];
  }
  a.n_parts = n_parts;
  a.mode = mode;
  a.n_px = n_px;
  a.out = map_out;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return amr::set_error(AMR_E_CUDA, cudaGetErrorString(e));
  const int block = 256;
  const int64_t want = (n_px + block - 1) / block;
  const int grid = (int)(want < (int64_t)sms * 8 ? want : (int64_t)sms * 8);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  if (precision == AMR_PREC_FP64) amr::merge_kernel<double><<<grid, block, 0, s>>>(a);
  else amr::merge_kernel<float><<<grid, block, 0, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return amr::set_error(AMR_E_CUDA, cudaGetErrorString(e));
  return AMR_OK;
}

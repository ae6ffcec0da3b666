// Adaptive Gaussian blur (Sec. 2.2): a post-process whose filter size follows
// how finely the mesh is resolved under each pixel, against the aliasing of
// coarse cells in images that mix refinement levels.  The local resolution of a pixel is the
// density-weighted mean level of the leaves its ray crossed (an
// AMR_MODE_LEVEL render of the same camera): cell edge h = 2^-level, Gaussian
// sigma = h / (2 pixel) in pixels, no blur below half a pixel.  The filter is
// separable: a row pass then a column pass, each output pixel using its own
// sigma, weights exp(-k^2 / (2 sigma^2)) for |k| <= floor(3 sigma + 0.5)
// (at most 64) renormalised over the samples inside the map.
#include <cuda_runtime.h>

#include "amr_internal.h"

namespace amr {
namespace {

constexpr int kMaxRadius = 64;

__device__ __forceinline__ float sigma_of(float level, float inv_pixel) {
  // 2^-level / (2 pixel)
  return 0.5f * exp2f(-level) * inv_pixel;
}

template <bool COLUMNS>
__global__ void __launch_bounds__(256) blur_pass(const float* __restrict__ in, const float* __restrict__ level,
                                                 float inv_pixel, float* __restrict__ out, int nx, int ny) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  if (x >= nx || y >= ny) return;
  const size_t p = (size_t)y * nx + x;
  const float sg = sigma_of(__ldg(&level[p]), inv_pixel);
  if (!(sg >= 0.5f)) {
    out[p] = __ldg(&in[p]);
    return;
  }
  const int R = min(kMaxRadius, (int)(3.0f * sg + 0.5f));
  const float g = -0.5f / (sg * sg);
  // The centre tap, then the pairs at +-k sharing one weight (one exponential
  // per pair: the special-function unit is this pass's narrowest resource).
  const int pos = COLUMNS ? y : x, len = COLUMNS ? ny : nx;
  const size_t stride = COLUMNS ? (size_t)nx : 1;
  float acc = __ldg(&in[p]), norm = 1.0f;
  for (int k = 1; k <= R; ++k) {
    const float wgt = __expf(g * (float)(k * k));
    if (pos - k >= 0) {
      acc = fmaf(wgt, __ldg(&in[p - k * stride]), acc);
      norm += wgt;
    }
    if (pos + k < len) {
      acc = fmaf(wgt, __ldg(&in[p + k * stride]), acc);
      norm += wgt;
    }
  }
  out[p] = acc / norm;
}

}  // namespace

cudaError_t launch_blur(const float* in, const float* level, double pixel, float* tmp, float* out, int nx, int ny,
                        cudaStream_t s) {
  if (nx <= 0 || ny <= 0) return cudaSuccess;
  const dim3 block(256), grid((nx + 255) / 256, ny);
  const float inv_pixel = (float)(1.0 / pixel);
  blur_pass<false><<<grid, block, 0, s>>>(in, level, inv_pixel, tmp, nx, ny);
  blur_pass<true><<<grid, block, 0, s>>>(tmp, level, inv_pixel, out, nx, ny);
  return cudaGetLastError();
}

}  // namespace amr

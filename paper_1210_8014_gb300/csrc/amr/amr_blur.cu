// Adaptive Gaussian blur (Sec. 2.2): a post-process whose filter size follows
// how finely the mesh is resolved under each pixel, against the aliasing of
// coarse cells in images that mix refinement levels.  The local resolution of a pixel is the
// density-weighted mean level of the leaves its ray crossed (an
// AMR_MODE_LEVEL render of the same camera): cell edge h = 2^-level, Gaussian
// sigma = h / (2 pixel) in pixels, no blur below half a pixel.  The filter is
// separable: a row pass then a column pass, each output pixel using its own
// sigma, weights exp(-k^2 / (2 sigma^2)) for |k| <= floor(3 sigma + 0.5)
// (at most 64) renormalised over the samples inside the map; the weights come
// from one exponential per pixel by a multiplicative recurrence.  The row pass
// reads its taps through L1 (32 consecutive pixels of a row per warp); the
// column pass stages 32-column tiles with their halo in shared memory.
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
  // Weights w_k = exp(g k^2) by the recurrence w_k = w_(k-1) r_(k-1),
  // r_k = r_(k-1) exp(2g), from one exponential per pixel: the relative error
  // of w_k grows like k^2 ulp (1e-4 at k = 64, where w_k < e^-4.5), which
  // moves a normalised output by under 1e-6 of the largest input.  The centre
  // tap, then the pairs at +-k sharing one weight.
  const int pos = COLUMNS ? y : x, len = COLUMNS ? ny : nx;
  const int stride = COLUMNS ? nx : 1;
  const float e1 = expf(g), q = e1 * e1;
  float w = 1.0f, ratio = e1;
  float acc = __ldg(&in[p]), norm = 1.0f;
  if (pos - R >= 0 && pos + R < len) {
    // Interior: every tap inside the map, no bounds checks.  Four pairs of
    // taps per iteration: their eight loads are independent of the weight
    // recurrence, so they are all in flight before the first is used.
    const float* lo = in + p;
    const float* hi = in + p;
    int k = 1;
    for (; k + 3 <= R; k += 4) {
      const float a0 = __ldg(lo - stride) + __ldg(hi + stride);
      const float a1 = __ldg(lo - 2 * stride) + __ldg(hi + 2 * stride);
      const float a2 = __ldg(lo - 3 * stride) + __ldg(hi + 3 * stride);
      const float a3 = __ldg(lo - 4 * stride) + __ldg(hi + 4 * stride);
      lo -= 4 * stride;
      hi += 4 * stride;
      w *= ratio;
      ratio *= q;
      acc = fmaf(w, a0, acc);
      norm = fmaf(2.0f, w, norm);
      w *= ratio;
      ratio *= q;
      acc = fmaf(w, a1, acc);
      norm = fmaf(2.0f, w, norm);
      w *= ratio;
      ratio *= q;
      acc = fmaf(w, a2, acc);
      norm = fmaf(2.0f, w, norm);
      w *= ratio;
      ratio *= q;
      acc = fmaf(w, a3, acc);
      norm = fmaf(2.0f, w, norm);
    }
    for (; k <= R; ++k) {
      w *= ratio;
      ratio *= q;
      lo -= stride;
      hi += stride;
      acc = fmaf(w, __ldg(lo) + __ldg(hi), acc);
      norm = fmaf(2.0f, w, norm);
    }
  } else {
    for (int k = 1; k <= R; ++k) {
      w *= ratio;
      ratio *= q;
      if (pos - k >= 0) {
        acc = fmaf(w, __ldg(&in[p - (size_t)k * stride]), acc);
        norm += w;
      }
      if (pos + k < len) {
        acc = fmaf(w, __ldg(&in[p + (size_t)k * stride]), acc);
        norm += w;
      }
    }
  }
  out[p] = acc / norm;
}

// The column pass on tiles of 32 columns x 64 rows staged in shared memory
// with 64 rows of halo above and below: a block of 32 x 8 threads, each
// thread 8 pixels of its column.  Every tap is a conflict-free shared load.
constexpr int kColTile = 64;
__global__ void __launch_bounds__(256) blur_cols_staged(const float* __restrict__ in, const float* __restrict__ level,
                                                        float inv_pixel, float* __restrict__ out, int nx, int ny) {
  __shared__ float tile[(kColTile + 2 * kMaxRadius) * 32];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int x = blockIdx.x * 32 + tx, y0 = blockIdx.y * kColTile;
  for (int r = ty; r < kColTile + 2 * kMaxRadius; r += 8) {
    const int gy = y0 - kMaxRadius + r;
    tile[r * 32 + tx] = (x < nx && gy >= 0 && gy < ny) ? __ldg(&in[(size_t)gy * nx + x]) : 0.0f;
  }
  __syncthreads();
  if (x >= nx) return;
  for (int i = 0; i < kColTile / 8; ++i) {
    const int yl = ty + 8 * i, y = y0 + yl;
    if (y >= ny) break;
    const float* t = tile + (yl + kMaxRadius) * 32 + tx;
    const size_t p = (size_t)y * nx + x;
    const float sg = sigma_of(__ldg(&level[p]), inv_pixel);
    if (!(sg >= 0.5f)) {
      out[p] = t[0];
      continue;
    }
    const int R = min(kMaxRadius, (int)(3.0f * sg + 0.5f));
    const float g = -0.5f / (sg * sg);
    const float e1 = expf(g), q = e1 * e1;
    float w = 1.0f, ratio = e1;
    float acc = t[0], norm = 1.0f;
    if (y - R >= 0 && y + R < ny) {
      int k = 1;
      for (; k + 3 <= R; k += 4) {
        const float a0 = t[-k * 32] + t[k * 32];
        const float a1 = t[(-k - 1) * 32] + t[(k + 1) * 32];
        const float a2 = t[(-k - 2) * 32] + t[(k + 2) * 32];
        const float a3 = t[(-k - 3) * 32] + t[(k + 3) * 32];
        w *= ratio;
        ratio *= q;
        acc = fmaf(w, a0, acc);
        norm = fmaf(2.0f, w, norm);
        w *= ratio;
        ratio *= q;
        acc = fmaf(w, a1, acc);
        norm = fmaf(2.0f, w, norm);
        w *= ratio;
        ratio *= q;
        acc = fmaf(w, a2, acc);
        norm = fmaf(2.0f, w, norm);
        w *= ratio;
        ratio *= q;
        acc = fmaf(w, a3, acc);
        norm = fmaf(2.0f, w, norm);
      }
      for (; k <= R; ++k) {
        w *= ratio;
        ratio *= q;
        acc = fmaf(w, t[-k * 32] + t[k * 32], acc);
        norm = fmaf(2.0f, w, norm);
      }
    } else {
      for (int k = 1; k <= R; ++k) {
        w *= ratio;
        ratio *= q;
        if (y - k >= 0) {
          acc = fmaf(w, t[-k * 32], acc);
          norm += w;
        }
        if (y + k < ny) {
          acc = fmaf(w, t[k * 32], acc);
          norm += w;
        }
      }
    }
    out[p] = acc / norm;
  }
}

}  // namespace

cudaError_t launch_blur(const float* in, const float* level, double pixel, float* tmp, float* out, int nx, int ny,
                        cudaStream_t s) {
  if (nx <= 0 || ny <= 0) return cudaSuccess;
  const dim3 block(256), grid((nx + 255) / 256, ny);
  const float inv_pixel = (float)(1.0 / pixel);
  blur_pass<false><<<grid, block, 0, s>>>(in, level, inv_pixel, tmp, nx, ny);
  blur_cols_staged<<<dim3((nx + 31) / 32, (ny + kColTile - 1) / kColTile), dim3(32, 8), 0, s>>>(tmp, level, inv_pixel, out,
                                                                                              nx, ny);
  return cudaGetLastError();
}

}  // namespace amr

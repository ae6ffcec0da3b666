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
// column pass stages 32-column tiles with their halo in shared memory.  Both
// passes are bound by instruction issue, so the interior sums run two taps
// at a time in packed FP32 pairs, and the per-pixel exponential and the two
// divisions use the hardware approximations (__expf, __fdividef: a few ulp,
// under 1e-6 of the output).
#include <cuda_runtime.h>

#include "amr_internal.h"

namespace amr {
namespace {

constexpr int kMaxRadius = 64;

__device__ __forceinline__ float sigma_of(float level, float inv_pixel) {
  // 2^-level / (2 pixel)
  return 0.5f * exp2f(-level) * inv_pixel;
}

// Interior sum over k = 1..R of w_k (x_-k + x_k), w_k = exp(g k^2) with
// e1 = exp(g), two k at a time in packed FP32 pairs: w_(k+2) = w_k rho_k with
// rho_k = exp(g (4k + 4)), and rho_(k+2) = rho_k exp(8g), so (w_k, w_(k+1))
// and (rho_k, rho_(k+1)) each advance by one packed multiply.  tap(k) returns
// x_-k + x_k.  Returns (sum of weighted taps, sum of weights).
template <typename Tap>
__device__ __forceinline__ float2 interior_pairs(int R, float e1, Tap tap) {
  const float q = e1 * e1;                 // exp(2g)
  float2 w = make_float2(e1, e1 * e1 * e1 * e1);  // (w_1, w_2) = (exp(g), exp(4g))
  const float Q = q * q;                   // exp(4g)
  float2 rho = make_float2(Q * Q, Q * Q * Q);     // (exp(8g), exp(12g)) = (w_3 / w_1, w_4 / w_2)
  const float2 QQ = make_float2(Q * Q, Q * Q);    // w_(k+2) / w_k = exp(g (4k + 4)) grows by exp(8g)
  float2 acc = make_float2(0.0f, 0.0f), ws = make_float2(0.0f, 0.0f);
  int k = 1;
  for (; k + 1 <= R; k += 2) {
    const float2 a = make_float2(tap(k), tap(k + 1));
    acc = __ffma2_rn(w, a, acc);
    ws = __fadd2_rn(ws, w);
    w = __fmul2_rn(w, rho);
    rho = __fmul2_rn(rho, QQ);
  }
  float s = acc.x + acc.y, n = ws.x + ws.y;
  if (k <= R) {  // odd R: the last k, whose weight is w.x
    s = fmaf(w.x, tap(k), s);
    n += w.x;
  }
  return make_float2(s, n);
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
  const float g = __fdividef(-0.5f, sg * sg);
  // Weights w_k = exp(g k^2) by multiplicative recurrences from one
  // exponential per pixel (pairs of k in the interior, w_k = w_(k-1) r_(k-1),
  // r_k = r_(k-1) exp(2g) at the map's edges): the relative error of w_k grows
  // like k^2 ulp (1e-4 at k = 64, where w_k < e^-4.5), which moves a
  // normalised output by under 1e-6 of the largest input.  The centre tap,
  // then the taps at +-k sharing one weight.
  const int pos = COLUMNS ? y : x, len = COLUMNS ? ny : nx;
  const int stride = COLUMNS ? nx : 1;
  const float e1 = __expf(g), q = e1 * e1;
  float w = 1.0f, ratio = e1;
  float acc = __ldg(&in[p]), norm = 1.0f;
  if (pos - R >= 0 && pos + R < len) {
    // Interior: every tap inside the map, no bounds checks.
    const float* c = in + p;
    const float2 sn = interior_pairs(R, e1, [&](int k) { return __ldg(c - k * stride) + __ldg(c + k * stride); });
    acc += sn.x;
    norm = fmaf(2.0f, sn.y, norm);
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
  out[p] = __fdividef(acc, norm);
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
    const float g = __fdividef(-0.5f, sg * sg);
    const float e1 = __expf(g), q = e1 * e1;
    float w = 1.0f, ratio = e1;
    float acc = t[0], norm = 1.0f;
    if (y - R >= 0 && y + R < ny) {
      const float2 sn = interior_pairs(R, e1, [&](int k) { return t[-k * 32] + t[k * 32]; });
      acc += sn.x;
      norm = fmaf(2.0f, sn.y, norm);
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
    out[p] = __fdividef(acc, norm);
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

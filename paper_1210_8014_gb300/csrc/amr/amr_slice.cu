// Slice map (Sec. 3.3: the slice-map tree search the authors ported to the
// GPU): for every pixel centre on the camera plane, the leaf holding
// that point at the camera's level cut.  One thread per pixel; the point is
// quantised exactly as a ray origin, and the descent reads the cell index of
// each level straight from the bits of the integer coordinates.
#include <cuda_runtime.h>

#include "amr.h"
#include "amr_internal.h"

namespace amr {
namespace {

constexpr long long kBoxS = 1LL << kFixBits;

template <bool OUT64, typename F>
__global__ void __launch_bounds__(256) slice_kernel(const uint2* __restrict__ rec, uint32_t n_oct,
                                                    const CamDev* __restrict__ camp, int32_t* __restrict__ err) {
  const CamDev& cam = *camp;
  const int64_t px = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (px >= (int64_t)cam.nx * cam.ny) return;
  const int i = (int)(px % cam.nx), j = (int)(px / cam.nx);
  long long X[3];
  if (cam.st) {  // per-camera column and row terms, rounded as below
    const double* col = cam.st + 3 * (size_t)i;
    const double* row = cam.st + 3 * ((size_t)cam.nx + j);
#pragma unroll
    for (int a = 0; a < 3; ++a) X[a] = __double2ll_rn(__dadd_rn(__ldg(col + a), __ldg(row + a)));
  } else {
    const double s = __dmul_rn(__dsub_rn(__ddiv_rn(__dadd_rn((double)i, 0.5), cam.nxd), 0.5), cam.fov0);
    const double t = __dmul_rn(__dsub_rn(__ddiv_rn(__dadd_rn((double)j, 0.5), cam.nyd), 0.5), cam.fov1);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double x = __dadd_rn(__dadd_rn(cam.centre[a], __dmul_rn(s, cam.u[a])), __dmul_rn(t, cam.v[a]));
      X[a] = __double2ll_rn(__dmul_rn(x, 68719476736.0 /* 2^36 */));
    }
  }
  bool inside = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) inside &= X[a] >= 0 && X[a] < kBoxS;
  double value = 0.0;
  int level = 0;
  if (inside) {
    uint32_t o = 0;
    uint2 r = __ldg(&rec[0]);
    for (int lvl = 1;; ++lvl) {
      const int sh = kFixBits - lvl;
      const int c = (int)((X[0] >> sh) & 1) | (int)(((X[1] >> sh) & 1) << 1) | (int)(((X[2] >> sh) & 1) << 2);
      if (!((r.y >> c) & 1u) || lvl >= cam.L) {
        value = (double)__ldg(static_cast<const F*>(cam.rho) + (size_t)o * 8 + c);
        level = lvl;
        break;
      }
      o = r.x + __popc(r.y & ((1u << c) - 1u));
      if (o >= n_oct || lvl >= kMaxLevel) {
        atomicExch(err, 1);
        break;
      }
      r = __ldg(&rec[o]);
    }
  }
  if (OUT64) static_cast<double*>(cam.map)[px] = value;
  else static_cast<float*>(cam.map)[px] = (float)value;
  if (cam.counts) cam.counts[px] = level;
}

}  // namespace

cudaError_t launch_slice(bool out64, bool f64, const uint2* rec, uint32_t n_oct, const CamDev* cam, int64_t n_px,
                         int32_t* err, cudaStream_t s) {
  const int block = 256;
  const int64_t grid = (n_px + block - 1) / block;
  if (grid <= 0) return cudaSuccess;
  if (out64) {
    if (f64) slice_kernel<true, double><<<(unsigned)grid, block, 0, s>>>(rec, n_oct, cam, err);
    else slice_kernel<true, float><<<(unsigned)grid, block, 0, s>>>(rec, n_oct, cam, err);
  } else {
    if (f64) slice_kernel<false, double><<<(unsigned)grid, block, 0, s>>>(rec, n_oct, cam, err);
    else slice_kernel<false, float><<<(unsigned)grid, block, 0, s>>>(rec, n_oct, cam, err);
  }
  return cudaGetLastError();
}

}  // namespace amr

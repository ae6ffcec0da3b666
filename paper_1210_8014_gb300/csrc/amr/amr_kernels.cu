// Launch functions of the octree-AMR ray casting kernels (the device code is
// in amr_trace.cuh): the batch kernels at the default register cap, the
// choice of kernel for a launch, and the gather that packs weighted-mean
// fields.
#include "amr_trace.cuh"

namespace amr {
namespace {

template <int PREC, bool NB, typename F, bool PARTIAL, int REGS>
const void* kernel_ptr() {
  return reinterpret_cast<const void*>(&batch_kernel<PREC, NB, F, PARTIAL, REGS>);
}

template <bool NB, typename F, bool PARTIAL, int REGS = kDefaultRegs>
const void* pick_prec(int prec) {
  switch (prec) {
    case AMR_PREC_FP64: return kernel_ptr<AMR_PREC_FP64, NB, F, PARTIAL, REGS>();
    case AMR_PREC_FP32_KAHAN: return kernel_ptr<AMR_PREC_FP32_KAHAN, NB, F, PARTIAL, REGS>();
    default: return kernel_ptr<AMR_PREC_FP32_PLAIN, NB, F, PARTIAL, REGS>();
  }
}

// nb: the launch carries face-neighbour links; partial: it stores accumulators
// (only launches with links do); regs: the register cap, which only the
// map-output kernels with links offer besides the default.
const void* pick(int prec, bool f64, bool nb, bool partial, int regs) {
  if (nb && partial) return f64 ? pick_prec<true, double, true>(prec) : pick_prec<true, float, true>(prec);
  if (nb) {
    if (regs != kDefaultRegs)
      if (const void* k = batch_kernel_capped(prec, f64, regs)) return k;
    return f64 ? pick_prec<true, double, false>(prec) : pick_prec<true, float, false>(prec);
  }
  return f64 ? pick_prec<false, double, false>(prec) : pick_prec<false, float, false>(prec);
}

template <typename F>
__global__ void __launch_bounds__(256) pack_kernel(const F* __restrict__ f0, const F* __restrict__ f1,
                                                   const F* __restrict__ f2, const F* __restrict__ f3, F* out,
                                                   int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    out[4 * i + 0] = f0[i];
    out[4 * i + 1] = f1[i];
    out[4 * i + 2] = f2[i];
    out[4 * i + 3] = f3[i];
  }
}

}  // namespace

cudaError_t launch_pack(bool f64, const void* f0, const void* f1, const void* f2, const void* f3, void* out,
                        int64_t n_cells, cudaStream_t s) {
  if (n_cells <= 0) return cudaSuccess;
  const int64_t blocks = (n_cells + 255) / 256;
  const int grid = (int)(blocks < 152 * 16 ? blocks : 152 * 16);
  if (f64)
    pack_kernel<double><<<grid, 256, 0, s>>>(static_cast<const double*>(f0), static_cast<const double*>(f1),
                                              static_cast<const double*>(f2), static_cast<const double*>(f3),
                                              static_cast<double*>(out), n_cells);
  else
    pack_kernel<float><<<grid, 256, 0, s>>>(static_cast<const float*>(f0), static_cast<const float*>(f1),
                                             static_cast<const float*>(f2), static_cast<const float*>(f3),
                                             static_cast<float*>(out), n_cells);
  return cudaGetLastError();
}

cudaError_t launch_batch(int prec, bool f64, const BatchArgs& a, int grid, int block, int regs, cudaStream_t s) {
  void* args[] = {const_cast<BatchArgs*>(&a)};
  return cudaLaunchKernel(pick(prec, f64, a.nbr != nullptr, a.partial != 0, regs), dim3(grid), dim3(block), args, 0,
                          s);
}

cudaError_t batch_occupancy(int prec, bool f64, bool nb, int block, int regs, int* blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, pick(prec, f64, nb, false, regs), block, 0);
}

int batch_regs(int prec, bool f64, bool nb, int regs) {
  cudaFuncAttributes at{};
  if (cudaFuncGetAttributes(&at, pick(prec, f64, nb, false, regs)) != cudaSuccess) return -1;
  return at.numRegs;
}

}  // namespace amr

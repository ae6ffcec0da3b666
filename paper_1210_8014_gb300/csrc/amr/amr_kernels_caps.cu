// The map-output batch kernels with face links at the register caps other
// than the default (56: 36 resident warps per SM with 128-thread blocks; 72:
// 28), compiled apart from amr_kernels.cu so that the two build in parallel.
#include "amr_trace.cuh"

namespace amr {
namespace {

template <int PREC, typename F, int REGS>
const void* capped_ptr() {
  return reinterpret_cast<const void*>(&batch_kernel<PREC, true, F, false, REGS>);
}

template <typename F, int REGS>
const void* capped_prec(int prec) {
  switch (prec) {
    case AMR_PREC_FP64: return capped_ptr<AMR_PREC_FP64, F, REGS>();
    case AMR_PREC_FP32_KAHAN: return capped_ptr<AMR_PREC_FP32_KAHAN, F, REGS>();
    default: return capped_ptr<AMR_PREC_FP32_PLAIN, F, REGS>();
  }
}

}  // namespace

const void* batch_kernel_capped(int prec, bool f64, int regs) {
  switch (regs) {
    case 56: return f64 ? capped_prec<double, 56>(prec) : capped_prec<float, 56>(prec);
    case 72: return f64 ? capped_prec<double, 72>(prec) : capped_prec<float, 72>(prec);
    default: return nullptr;
  }
}

}  // namespace amr

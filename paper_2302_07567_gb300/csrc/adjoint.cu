// Adjoint of the FMM operator (placeholder until the adjoint kernels land).
#include "common.cuh"

namespace fmm {
int run_adjoint(fmm_plan_s*, const double*, const double*, const double*, const void*, const void*, double*,
                double*, double*, cudaStream_t) {
  return FMM_EINVAL;
}
}  // namespace fmm

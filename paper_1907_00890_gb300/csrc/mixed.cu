// Mixed-precision path (FP32 transforms, FP64 low modes, residual and reductions, defect correction).
#include "passes.cuh"
#include "solve_internal.h"

namespace vofp {

void init_kernel_attributes_mixed() {}

int mixed_solve(vofp_plan*, int, const XArgs*, const double*, double*, cudaStream_t, vofp_info*) {
  return VOFP_ERR_UNSUPPORTED;
}

}  // namespace vofp

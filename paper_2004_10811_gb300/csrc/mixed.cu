// Mixed-precision path and adjoint (filled in by the tensor-core kernels).
#include "plan.cuh"

namespace submat {

size_t mixed_bytes_per_elem() { return 3 * 8; }

submat_status Plan::sign_mixed(const double*, double, double*, cudaStream_t) {
  set_error("mixed precision path not built yet");
  return SUBMAT_ERR_UNSUPPORTED;
}

submat_status Plan::backward(const double*, double, const double*, double*, double*, cudaStream_t) {
  set_error("adjoint not built yet");
  return SUBMAT_ERR_UNSUPPORTED;
}

}  // namespace submat

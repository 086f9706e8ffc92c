// Instantiation of the fused step kernel for bf16 population storage.
#include "step_kernel.cuh"

namespace pflbm {
cudaError_t launch_step_bf16(int form, const StepArgs& a, cudaStream_t s) {
  return launch_step_impl<StoreBF16>(form, a, s);
}
}  // namespace pflbm

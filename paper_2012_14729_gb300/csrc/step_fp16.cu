// Instantiation of the fused step kernel for fp16 population storage.
#include "step_kernel.cuh"

namespace pflbm {
cudaError_t launch_step_fp16(int form, const StepArgs& a, cudaStream_t s) {
  return launch_step_impl<StoreF16>(form, a, s);
}
}  // namespace pflbm

// Instantiation of the fused step kernel for fp32 population storage.
#include "step_kernel.cuh"

namespace pflbm {
cudaError_t launch_step_fp32(int form, const StepArgs& a, cudaStream_t s) {
  return launch_step_impl<StoreF32>(form, a, s);
}
}  // namespace pflbm

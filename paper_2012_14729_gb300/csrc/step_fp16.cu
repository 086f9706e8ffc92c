// Instantiation of the fused step kernels for fp16 population storage.
#include "march_kernel.cuh"

namespace pflbm {
cudaError_t launch_step_fp16(int form, int mode, const StepArgs& a, cudaStream_t s) {
  return launch_step_impl<StoreF16>(form, mode, a, s);
}
}  // namespace pflbm

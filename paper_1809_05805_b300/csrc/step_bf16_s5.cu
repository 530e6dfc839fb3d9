// Instantiations of the one-reduce step kernel: FP32 arithmetic on a BF16 basis, staged CSR, tile pairs without the column ring.
#include "step.cuh"

namespace lsg_steps {
const void* step_kernel_bf16_s5(int m) {
  return reinterpret_cast<const void*>(step_kernel_staged<float, __nv_bfloat16, 5>(m));
}
}  // namespace lsg_steps

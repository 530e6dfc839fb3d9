// Instantiations of the one-reduce step kernel: FP32 arithmetic and basis, staged CSR, tile pairs without the column ring.
#include "step.cuh"

namespace lsg_steps {
const void* step_kernel_f32_s5(int m) {
  return reinterpret_cast<const void*>(step_kernel_staged<float, float, 5>(m));
}
}  // namespace lsg_steps

// Instantiations of the one-reduce step kernel: FP32 arithmetic and basis, CSR read from global memory.
#include "step.cuh"

namespace lsg_steps {
const void* step_kernel_f32_s0(int m) {
  return reinterpret_cast<const void*>(step_kernel_staged<float, float, 0>(m));
}
}  // namespace lsg_steps

// Instantiations of the one-reduce step kernel: FP64, staged CSR, tile pairs
// with the column ring, block dot on the integer pipes (fixed-point products).
#include "step.cuh"

namespace lsg_steps {
const void* step_kernel_f64_s6(int m) {
  return reinterpret_cast<const void*>(step_kernel_staged<double, double, 6>(m));
}
}  // namespace lsg_steps

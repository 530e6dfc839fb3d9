// Instantiations of the one-reduce step kernel: FP64 arithmetic and basis, staged CSR, tile pairs without the column ring.
#include "step.cuh"

namespace lsg_steps {
const void* step_kernel_f64_s5(int m) {
  return reinterpret_cast<const void*>(step_kernel_staged<double, double, 5>(m));
}
}  // namespace lsg_steps

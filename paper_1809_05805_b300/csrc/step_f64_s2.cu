// Instantiations of the one-reduce step kernel: FP64 arithmetic and basis, staged CSR, tile pairs.
#include "step.cuh"

namespace lsg_steps {
const void* step_kernel_f64_s2(int m) {
  return reinterpret_cast<const void*>(step_kernel_staged<double, double, 2>(m));
}
}  // namespace lsg_steps

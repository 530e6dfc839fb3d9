// Instantiations of the one-reduce step kernel: FP64 arithmetic and basis, staged CSR, one tile per unit.
#include "step.cuh"

namespace lsg_steps {
const void* step_kernel_f64_s1(int m) {
  return reinterpret_cast<const void*>(step_kernel_staged<double, double, 1>(m));
}
}  // namespace lsg_steps

// Instantiations of the engine step kernel with float arithmetic.
#include "engine_step.cuh"

namespace lsg_engine {
const void* eng_step_f32(int m, bool pairs, int fx) {
  return reinterpret_cast<const void*>(eng_step_table<float>(m, pairs, fx));
}
}  // namespace lsg_engine

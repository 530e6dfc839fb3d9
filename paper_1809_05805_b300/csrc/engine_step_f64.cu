// Instantiations of the engine step kernel with double arithmetic.
#include "engine_step.cuh"

namespace lsg_engine {
const void* eng_step_f64(int m, bool pairs, int fx) {
  return reinterpret_cast<const void*>(eng_step_table<double>(m, pairs, fx));
}
}  // namespace lsg_engine

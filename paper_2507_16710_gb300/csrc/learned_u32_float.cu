// learned_u32_float.cu -- learned-CDF bucketing path for 32-bit float keys.
#include "learned_launch.cuh"

namespace ak {
cudaError_t learned_launch_u32_float(const RadixCall &c, const LearnedCall &lc) {
  return learned_launch<uint32_t, KIND_FLOAT>(c, lc);
}
}  // namespace ak

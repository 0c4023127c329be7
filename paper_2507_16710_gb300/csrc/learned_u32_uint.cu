// learned_u32_uint.cu -- learned-CDF bucketing path for 32-bit uint keys.
#include "learned_launch.cuh"

namespace ak {
cudaError_t learned_launch_u32_uint(const RadixCall &c, const LearnedCall &lc) {
  return learned_launch<uint32_t, KIND_UINT>(c, lc);
}
}  // namespace ak

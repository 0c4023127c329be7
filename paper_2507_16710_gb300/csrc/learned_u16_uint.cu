// learned_u16_uint.cu -- learned-CDF bucketing path for 16-bit uint keys.
#include "learned_launch.cuh"

namespace ak {
cudaError_t learned_launch_u16_uint(const RadixCall &c, const LearnedCall &lc) {
  return learned_launch<uint16_t, KIND_UINT>(c, lc);
}
}  // namespace ak

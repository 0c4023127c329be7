// learned_u64_uint.cu -- learned-CDF bucketing path for 64-bit uint keys.
#include "learned_launch.cuh"

namespace ak {
cudaError_t learned_launch_u64_uint(const RadixCall &c, const LearnedCall &lc) {
  return learned_launch<uint64_t, KIND_UINT>(c, lc);
}
}  // namespace ak

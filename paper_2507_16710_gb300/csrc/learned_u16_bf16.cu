// learned_u16_bf16.cu -- learned-CDF bucketing path for bfloat16 keys.
#include "learned_launch.cuh"

namespace ak {
cudaError_t learned_launch_u16_bf16(const RadixCall &c, const LearnedCall &lc) {
  return learned_launch<uint16_t, KIND_BF16>(c, lc);
}
}  // namespace ak

// learned_u32_sint.cu -- learned-CDF bucketing path for 32-bit sint keys.
#include "learned_launch.cuh"

namespace ak {
cudaError_t learned_launch_u32_sint(const RadixCall &c, const LearnedCall &lc) {
  return learned_launch<uint32_t, KIND_SINT>(c, lc);
}
}  // namespace ak

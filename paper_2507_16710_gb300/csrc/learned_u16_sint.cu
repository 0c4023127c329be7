// learned_u16_sint.cu -- learned-CDF bucketing path for 16-bit sint keys.
#include "learned_launch.cuh"

namespace ak {
cudaError_t learned_launch_u16_sint(const RadixCall &c, const LearnedCall &lc) {
  return learned_launch<uint16_t, KIND_SINT>(c, lc);
}
}  // namespace ak

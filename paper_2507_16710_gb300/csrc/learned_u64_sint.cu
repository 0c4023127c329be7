// learned_u64_sint.cu -- learned-CDF bucketing path for 64-bit sint keys.
#include "learned_launch.cuh"

namespace ak {
cudaError_t learned_launch_u64_sint(const RadixCall &c, const LearnedCall &lc) {
  return learned_launch<uint64_t, KIND_SINT>(c, lc);
}
}  // namespace ak

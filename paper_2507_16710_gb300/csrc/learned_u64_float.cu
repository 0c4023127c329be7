// learned_u64_float.cu -- learned-CDF bucketing path for 64-bit float keys.
#include "learned_launch.cuh"

namespace ak {
cudaError_t learned_launch_u64_float(const RadixCall &c, const LearnedCall &lc) {
  return learned_launch<uint64_t, KIND_FLOAT>(c, lc);
}
}  // namespace ak

// learned_u16_float.cu -- learned-CDF bucketing path for 16-bit IEEE float (binary16) keys.
#include "learned_launch.cuh"

namespace ak {
cudaError_t learned_launch_u16_float(const RadixCall &c, const LearnedCall &lc) {
  return learned_launch<uint16_t, KIND_FLOAT>(c, lc);
}
}  // namespace ak

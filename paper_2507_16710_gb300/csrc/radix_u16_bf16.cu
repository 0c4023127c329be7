// radix_u16_bf16.cu -- onesweep radix sort instantiated for bfloat16 keys.
#include "radix_launch.cuh"

namespace ak {
cudaError_t radix_launch_u16_bf16(const RadixCall &c) { return radix_launch<uint16_t, KIND_BF16>(c); }
}  // namespace ak

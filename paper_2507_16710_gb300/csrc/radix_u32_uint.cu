// radix_u32_uint.cu -- onesweep radix sort instantiated for 32-bit uint keys.
#include "radix_launch.cuh"

namespace ak {
cudaError_t radix_launch_u32_uint(const RadixCall &c) { return radix_launch<uint32_t, KIND_UINT>(c); }
}  // namespace ak

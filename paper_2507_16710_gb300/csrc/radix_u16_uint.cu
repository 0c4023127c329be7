// radix_u16_uint.cu -- onesweep radix sort instantiated for 16-bit uint keys.
#include "radix_launch.cuh"

namespace ak {
cudaError_t radix_launch_u16_uint(const RadixCall &c) { return radix_launch<uint16_t, KIND_UINT>(c); }
}  // namespace ak

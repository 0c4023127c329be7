// radix_u128_uint.cu -- onesweep radix sort instantiated for 128-bit uint keys.
#include "radix_launch.cuh"

namespace ak {
cudaError_t radix_launch_u128_uint(const RadixCall &c) { return radix_launch<u128, KIND_UINT>(c); }
}  // namespace ak

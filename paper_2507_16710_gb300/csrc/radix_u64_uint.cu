// radix_u64_uint.cu -- onesweep radix sort instantiated for 64-bit uint keys.
#include "radix_launch.cuh"

namespace ak {
cudaError_t radix_launch_u64_uint(const RadixCall &c) { return radix_launch<uint64_t, KIND_UINT>(c); }
}  // namespace ak

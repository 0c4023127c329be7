// radix_u32_sint.cu -- onesweep radix sort instantiated for 32-bit sint keys.
#include "radix_launch.cuh"

namespace ak {
cudaError_t radix_launch_u32_sint(const RadixCall &c) { return radix_launch<uint32_t, KIND_SINT>(c); }
}  // namespace ak

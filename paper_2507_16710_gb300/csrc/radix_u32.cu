// radix_u32.cu -- onesweep radix sort instantiated for 32-bit key words.
#include "radix_launch.cuh"

namespace ak {
cudaError_t radix_launch_u32(const RadixCall &c) { return radix_launch<uint32_t>(c); }
}  // namespace ak

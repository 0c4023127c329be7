// radix_u16.cu -- onesweep radix sort instantiated for 16-bit key words.
#include "radix_launch.cuh"

namespace ak {
cudaError_t radix_launch_u16(const RadixCall &c) { return radix_launch<uint16_t>(c); }
}  // namespace ak

// radix_u64.cu -- onesweep radix sort instantiated for 64-bit key words.
#include "radix_launch.cuh"

namespace ak {
cudaError_t radix_launch_u64(const RadixCall &c) { return radix_launch<uint64_t>(c); }
}  // namespace ak

// radix_u64_sint.cu -- onesweep radix sort instantiated for 64-bit sint keys.
#include "radix_launch.cuh"

namespace ak {
cudaError_t radix_launch_u64_sint(const RadixCall &c) { return radix_launch<uint64_t, KIND_SINT>(c); }
}  // namespace ak

// radix_u128_sint.cu -- onesweep radix sort instantiated for 128-bit sint keys.
#include "radix_launch.cuh"

namespace ak {
cudaError_t radix_launch_u128_sint(const RadixCall &c) { return radix_launch<u128, KIND_SINT>(c); }
}  // namespace ak

// radix_u16_sint.cu -- onesweep radix sort instantiated for 16-bit sint keys.
#include "radix_launch.cuh"

namespace ak {
cudaError_t radix_launch_u16_sint(const RadixCall &c) { return radix_launch<uint16_t, KIND_SINT>(c); }
}  // namespace ak

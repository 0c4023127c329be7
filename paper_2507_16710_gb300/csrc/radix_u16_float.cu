// radix_u16_float.cu -- onesweep radix sort instantiated for 16-bit IEEE float (binary16) keys.
#include "radix_launch.cuh"

namespace ak {
cudaError_t radix_launch_u16_float(const RadixCall &c) { return radix_launch<uint16_t, KIND_FLOAT>(c); }
}  // namespace ak

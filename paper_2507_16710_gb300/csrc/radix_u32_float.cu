// radix_u32_float.cu -- onesweep radix sort instantiated for 32-bit float keys.
#include "radix_launch.cuh"

namespace ak {
cudaError_t radix_launch_u32_float(const RadixCall &c) { return radix_launch<uint32_t, KIND_FLOAT>(c); }
}  // namespace ak

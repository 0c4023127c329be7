// radix_u64_float.cu -- onesweep radix sort instantiated for 64-bit float keys.
#include "radix_launch.cuh"

namespace ak {
cudaError_t radix_launch_u64_float(const RadixCall &c) { return radix_launch<uint64_t, KIND_FLOAT>(c); }
}  // namespace ak

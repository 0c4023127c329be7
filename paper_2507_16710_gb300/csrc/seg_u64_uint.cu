// seg_u64_uint.cu -- segmented sort instantiated for 64-bit uint keys.
#include "seg_launch.cuh"

namespace ak {
cudaError_t seg_launch_u64_uint(const SegCall &c) { return seg_launch<uint64_t, KIND_UINT>(c); }
}  // namespace ak

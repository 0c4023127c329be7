// seg_u32_uint.cu -- segmented sort instantiated for 32-bit uint keys.
#include "seg_launch.cuh"

namespace ak {
cudaError_t seg_launch_u32_uint(const SegCall &c) { return seg_launch<uint32_t, KIND_UINT>(c); }
}  // namespace ak

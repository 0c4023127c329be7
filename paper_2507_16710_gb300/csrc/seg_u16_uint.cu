// seg_u16_uint.cu -- segmented sort instantiated for 16-bit uint keys.
#include "seg_launch.cuh"

namespace ak {
cudaError_t seg_launch_u16_uint(const SegCall &c) { return seg_launch<uint16_t, KIND_UINT>(c); }
}  // namespace ak

// seg_u32_sint.cu -- segmented sort instantiated for 32-bit sint keys.
#include "seg_launch.cuh"

namespace ak {
cudaError_t seg_launch_u32_sint(const SegCall &c) { return seg_launch<uint32_t, KIND_SINT>(c); }
}  // namespace ak

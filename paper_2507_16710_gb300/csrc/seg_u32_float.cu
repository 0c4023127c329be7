// seg_u32_float.cu -- segmented sort instantiated for 32-bit float keys.
#include "seg_launch.cuh"

namespace ak {
cudaError_t seg_launch_u32_float(const SegCall &c) { return seg_launch<uint32_t, KIND_FLOAT>(c); }
}  // namespace ak

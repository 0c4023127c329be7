// seg_u16_sint.cu -- segmented sort instantiated for 16-bit sint keys.
#include "seg_launch.cuh"

namespace ak {
cudaError_t seg_launch_u16_sint(const SegCall &c) { return seg_launch<uint16_t, KIND_SINT>(c); }
}  // namespace ak

// seg_u16_float.cu -- segmented sort instantiated for 16-bit IEEE float (binary16) keys.
#include "seg_launch.cuh"

namespace ak {
cudaError_t seg_launch_u16_float(const SegCall &c) { return seg_launch<uint16_t, KIND_FLOAT>(c); }
}  // namespace ak

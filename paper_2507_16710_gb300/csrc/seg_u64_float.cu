// seg_u64_float.cu -- segmented sort instantiated for 64-bit float keys.
#include "seg_launch.cuh"

namespace ak {
cudaError_t seg_launch_u64_float(const SegCall &c) { return seg_launch<uint64_t, KIND_FLOAT>(c); }
}  // namespace ak

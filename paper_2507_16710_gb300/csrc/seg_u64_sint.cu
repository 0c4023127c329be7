// seg_u64_sint.cu -- segmented sort instantiated for 64-bit sint keys.
#include "seg_launch.cuh"

namespace ak {
cudaError_t seg_launch_u64_sint(const SegCall &c) { return seg_launch<uint64_t, KIND_SINT>(c); }
}  // namespace ak

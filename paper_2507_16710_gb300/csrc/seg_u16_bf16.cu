// seg_u16_bf16.cu -- segmented sort instantiated for bfloat16 keys.
#include "seg_launch.cuh"

namespace ak {
cudaError_t seg_launch_u16_bf16(const SegCall &c) { return seg_launch<uint16_t, KIND_BF16>(c); }
}  // namespace ak

// static_scratch.cu -- ak_sort with a built-in workspace, for callers that
// cannot allocate device memory.
//
// The workspace is a file-scope device array.  Every GPU that loads this library
// holds AK_STATIC_SCRATCH_BYTES of it until the process exits.  In host code the
// array's name is only a host-side stand-in, so its device address is looked up
// once per device with cudaGetSymbolAddress (with that device current) and
// cached; kernels are always given that address.
#include <mutex>

#include "internal.h"

static __device__ __align__(256) unsigned char g_static_scratch[AK_STATIC_SCRATCH_BYTES];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_static_scratch on the current device (set up on first use).
ak_status static_scratch_address(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return AK_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) return AK_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return AK_OK;
}

}  // namespace

extern "C" ak_status ak_sort_static_scratch(void *d_keys, int64_t n, ak_dtype kd, ak_order order,
                                            ak_stream_t stream) {
  if (n == 0) return ak_sort(d_keys, n, kd, order, nullptr, 0, stream, nullptr);
  size_t need = 0;
  const ak_status st = ak_sort_temp_bytes(AK_OP_SORT, n, kd, 0, 0, nullptr, &need);
  if (st != AK_OK) return st;
  if (need > size_t(AK_STATIC_SCRATCH_BYTES)) return AK_ERR_WORKSPACE_TOO_SMALL;
  void *scratch = nullptr;
  const ak_status a = static_scratch_address(&scratch);
  if (a != AK_OK) return a;
  return ak_sort(d_keys, n, kd, order, scratch, size_t(AK_STATIC_SCRATCH_BYTES), stream, nullptr);
}

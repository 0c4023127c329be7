// pending.cu -- entry points whose kernels are not built yet; each returns
// AK_ERR_UNSUPPORTED.
#include "internal.h"

extern "C" {
ak_status ak_autotune(int, int64_t, ak_dtype, int, ak_order, void *, void *, uint32_t *, void *, size_t,
                      ak_stream_t, ak_options *) {
  return AK_ERR_UNSUPPORTED;
}
ak_status ak_autotune_save(const char *) { return AK_ERR_UNSUPPORTED; }
ak_status ak_autotune_load(const char *) { return AK_ERR_UNSUPPORTED; }
void ak_autotune_clear(void) {}
}

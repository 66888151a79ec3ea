// Entry points whose kernels are not built yet.
#include "fw_internal.h"

extern "C" {
fw_status fw_backward(const float*, const float*, const int32_t*, float*, int64_t, int64_t, void*) {
  return FW_ERR_UNSUPPORTED;
}
fw_status fw_backward_strided(const float*, const float*, const int32_t*, float*, int64_t, int64_t,
                              int64_t, int64_t, void*) {
  return FW_ERR_UNSUPPORTED;
}
}

// Entry points whose kernels are not built yet.
#include "fw_internal.h"

extern "C" {
fw_status fw_batched_plan_create(fw_batched_plan** plan, const int64_t*, const int64_t*, int64_t,
                                 fw_dtype, const fw_options*) {
  if (plan) *plan = nullptr;
  return FW_ERR_UNSUPPORTED;
}
fw_status fw_solve_batched(fw_batched_plan*, void* const*, int32_t* const*, void*) {
  return FW_ERR_UNSUPPORTED;
}
fw_status fw_batched_plan_info(const fw_batched_plan*, int32_t*, int64_t*) { return FW_ERR_UNSUPPORTED; }
fw_status fw_batched_plan_destroy(fw_batched_plan*) { return FW_OK; }
fw_status fw_backward(const float*, const float*, const int32_t*, float*, int64_t, int64_t, void*) {
  return FW_ERR_UNSUPPORTED;
}
fw_status fw_backward_strided(const float*, const float*, const int32_t*, float*, int64_t, int64_t,
                              int64_t, int64_t, void*) {
  return FW_ERR_UNSUPPORTED;
}
}

// batched.cu -- ragged batches (placeholder until the persistent kernel lands).
#include "internal.h"

using namespace giga;

extern "C" {
giga_status_t giga_batched_plan_create(const giga_image_t*, int32_t, int32_t, int32_t, int32_t,
                                       giga_batched_plan_t* plan) {
  if (plan) *plan = nullptr;
  return fail(GIGA_ERR_UNSUPPORTED, "batched path not built");
}
giga_status_t giga_batched_plan_workspace_size(giga_batched_plan_t, size_t* bytes) {
  if (bytes) *bytes = 0;
  return fail(GIGA_ERR_UNSUPPORTED, "batched path not built");
}
giga_status_t giga_batched_plan_upload(giga_batched_plan_t, void*, size_t, void*) {
  return fail(GIGA_ERR_UNSUPPORTED, "batched path not built");
}
giga_status_t giga_batched_plan_run(giga_batched_plan_t, void*, size_t, void*) {
  return fail(GIGA_ERR_UNSUPPORTED, "batched path not built");
}
void giga_batched_plan_destroy(giga_batched_plan_t) {}
giga_status_t giga_conv2d_batched(const giga_image_t*, int32_t, int32_t, int32_t, int32_t, void*,
                                  size_t, void*) {
  return fail(GIGA_ERR_UNSUPPORTED, "batched path not built");
}
giga_status_t giga_conv2d_batched_workspace_size(const giga_image_t*, int32_t, int32_t,
                                                 size_t* bytes) {
  if (bytes) *bytes = 0;
  return fail(GIGA_ERR_UNSUPPORTED, "batched path not built");
}
}

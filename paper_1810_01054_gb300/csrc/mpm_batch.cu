// Batched scene execution (include/mpm.h, mpm_batch_*).
#include "../../include/mpm.h"

extern "C" {
mpm_status mpm_batch_create(mpm_ctx*, int, size_t, mpm_batch** out) {
  if (out) *out = nullptr;
  return MPM_ERR_STATE;
}
mpm_status mpm_batch_destroy(mpm_batch*) { return MPM_ERR_STATE; }
mpm_status mpm_batch_admit(mpm_batch*, mpm_scene*, int, int, int* slot) {
  if (slot) *slot = -1;
  return MPM_ERR_STATE;
}
mpm_status mpm_batch_tick(mpm_batch*, int) { return MPM_ERR_STATE; }
mpm_status mpm_batch_poll(mpm_batch*, int, int*) { return MPM_ERR_STATE; }
mpm_status mpm_batch_release(mpm_batch*, int) { return MPM_ERR_STATE; }
}

// Batched FISTA (placeholder until the persistent kernel lands).
#include "fm_internal.h"

struct fm_batch_s {
  int dummy;
};

extern "C" {
fm_status fm_batch_create(const fm_op*, int64_t, void*, fm_batch* out) {
  if (out) *out = nullptr;
  fm::set_error("batched FISTA is not built yet");
  return FM_ERR_UNSUPPORTED;
}
void fm_batch_release(fm_batch) {}
fm_status fm_batch_sizes(fm_batch, int64_t*, int64_t*) { return FM_ERR_UNSUPPORTED; }
fm_status fm_fista(fm_batch, const float*, float*, const fm_fista_params*, const fm_fista_report*, void*) {
  return FM_ERR_UNSUPPORTED;
}
}

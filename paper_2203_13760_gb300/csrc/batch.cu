// Batched simulations (placeholder until the persistent kernel lands).
#include "jf_internal.h"

namespace jf {
jf_status batch_set_variant(jf_ctx* h, int) { set_error(h, "batch: not built"); return JF_ERR_UNSUPPORTED; }
int batch_variant_info(jf_ctx*, int, char*, int) { return JF_ERR_UNSUPPORTED; }
}  // namespace jf

using namespace jf;
extern "C" {
jf_status jf_batch_create(const jf_grid*, int, const jf_gas*, const jf_scheme*, jf_handle* out) {
  if (out) *out = nullptr;
  set_error(nullptr, "jf_batch_create: not built yet");
  return JF_ERR_UNSUPPORTED;
}
jf_status jf_batch_step(jf_handle h, void* const*, int, double*, void*) {
  set_error(h, "jf_batch_step: not built yet");
  return JF_ERR_UNSUPPORTED;
}
}

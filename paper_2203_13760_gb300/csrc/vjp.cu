// Adjoint of the RK3 step (placeholder until the VJP kernels land).
#include "jf_internal.h"

using namespace jf;
extern "C" {
jf_status jf_rk3_step_vjp(jf_handle h, const void*, const double*, const void*, void*, void*) {
  set_error(h, "jf_rk3_step_vjp: not built yet");
  return JF_ERR_UNSUPPORTED;
}
}

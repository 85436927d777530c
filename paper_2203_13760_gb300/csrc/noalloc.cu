// jf_rk3_step_noalloc: one RK3 step without a handle and without any device
// memory allocation.
//
// Who needs it: callers that must not call cudaMalloc / cudaFree at run time,
// for example code that runs under a memory budget fixed at start-up, a host
// application whose allocator owns all device memory, or a step embedded in
// someone else's hot loop where an allocation (and the implicit device
// synchronisation cudaFree brings) is not acceptable.  jf_init allocates the
// stage buffers; this entry point uses a fixed scratch area instead.
//
// The scratch is the file-scope device array below, JF_NOALLOC_MAX_CELLS
// cells large for both stage buffers in FP64 (about 5.2 MB).  Every GPU that
// loads libjf holds it until the process exits.  All calls share it: calls
// whose work overlaps on the GPU (different streams, or different host
// threads, on one device) race on it and must be serialised by the caller.
#include <mutex>

#include "jf_internal.h"

namespace jf {
namespace {

constexpr long long kMaxCells = JF_NOALLOC_MAX_CELLS;  // include/jf.h
constexpr size_t kHeader = 256;  // reduction scratch, dt, error flag
constexpr size_t kStageBytes = 5 * (size_t)kMaxCells * sizeof(double);
constexpr size_t kScratchBytes = kHeader + 2 * kStageBytes;
constexpr size_t kRedOffset = 0, kDtOffset = 64, kFlagOffset = 128;
constexpr int kMaxDevices = 64;

// Device scratch of jf_rk3_step_noalloc.  In host code this name is only a
// host-side stand-in for the symbol; its device address comes from
// cudaGetSymbolAddress (see device_scratch).
__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct DeviceScratch {
  bool ready = false;
  unsigned char* base = nullptr;
  int sms = 1;
};
std::mutex g_mu;
DeviceScratch g_devices[kMaxDevices];

template <typename T>
cudaError_t prepare_all() {
  int count = 0;
  const StageVariant<T>* tab = stage_variants<T>(&count);
  for (int i = 0; i < count; ++i) {
    cudaError_t e = tab[i].prepare();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Once per device, with that device current: resolve the scratch array's
// device address and set the kernels' shared-memory attributes.
jf_status device_scratch(int dev, DeviceScratch** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (dev < 0 || dev >= kMaxDevices) {
    set_error(nullptr, "jf_rk3_step_noalloc: device index out of range");
    return JF_ERR_UNSUPPORTED;
  }
  DeviceScratch& d = g_devices[dev];
  if (!d.ready) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "jf_rk3_step_noalloc: cudaGetSymbolAddress");
    e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "jf_rk3_step_noalloc: device query");
    if ((e = prepare_all<float>()) != cudaSuccess || (e = prepare_all<double>()) != cudaSuccess)
      return cuda_fail(nullptr, e, "jf_rk3_step_noalloc: cudaFuncSetAttribute");
    d.base = static_cast<unsigned char*>(p);
    d.ready = true;
  }
  *out = &d;
  return JF_OK;
}

}  // namespace
}  // namespace jf

using namespace jf;

extern "C" jf_status jf_rk3_step_noalloc(const jf_grid* grid, const jf_gas* gas, const jf_scheme* scheme,
                                         void* U_inout, const double* dt_dev, double* dt_used_dev, void* stream) {
  if (!grid || !gas || !scheme || !U_inout || !aligned16(U_inout)) {
    set_error(nullptr, "jf_rk3_step_noalloc: null or misaligned argument");
    return JF_ERR_ARG;
  }
  jf_status st;
  if ((st = check_grid(nullptr, *grid)) != JF_OK) return st;
  if ((st = check_physics(nullptr, *gas, *scheme)) != JF_OK) return st;
  if (scheme->flux == JF_FLUX_RUSANOV_NN) {
    set_error(nullptr, "jf_rk3_step_noalloc: the Rusanov-NN flux needs a handle (jf_set_nn)");
    return JF_ERR_UNSUPPORTED;
  }
  const long long cells = (long long)grid->nx * grid->ny * grid->nz;
  if (cells > kMaxCells) {
    set_error(nullptr, "jf_rk3_step_noalloc: the grid has more cells than the fixed scratch holds "
                       "(JF_NOALLOC_MAX_CELLS = 65536); use jf_init / jf_rk3_step");
    return JF_ERR_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "jf_rk3_step_noalloc: cudaGetDevice");
  DeviceScratch* d = nullptr;
  if ((st = device_scratch(dev, &d)) != JF_OK) return st;

  // A handle on the stack whose buffers all point into the scratch array.
  jf_ctx h;
  h.kind = 0;
  h.grid = *grid;
  h.gas = *gas;
  h.scheme = *scheme;
  h.dim = active_dims(*grid);
  h.esize = scheme->dtype == JF_F32 ? 4 : 8;
  h.N = (size_t)cells;
  h.device = dev;
  h.sms = d->sms;
  h.red_cfl = reinterpret_cast<ReduceScratch*>(d->base + kRedOffset);
  h.dt_buf = reinterpret_cast<double*>(d->base + kDtOffset);
  h.flag = reinterpret_cast<int*>(d->base + kFlagOffset);
  h.stage[0] = d->base + kHeader;
  h.stage[1] = d->base + kHeader + kStageBytes;
  // the array keeps the previous call's contents: the reduction accumulator
  // and ticket must start at zero
  e = cudaMemsetAsync(d->base, 0, kHeader, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "jf_rk3_step_noalloc: cudaMemsetAsync");
  st = scheme->dtype == JF_F32 ? select_variant<float>(&h, -1, false) : select_variant<double>(&h, -1, false);
  if (st == JF_OK)
    st = scheme->dtype == JF_F32 ? step_impl<float>(&h, U_inout, dt_dev, dt_used_dev, (cudaStream_t)stream)
                                 : step_impl<double>(&h, U_inout, dt_dev, dt_used_dev, (cudaStream_t)stream);
  if (st != JF_OK) set_error(nullptr, h.err);
  // nothing of h is released: its buffers belong to the scratch array
  h.stage[0] = h.stage[1] = nullptr;
  return st;
}

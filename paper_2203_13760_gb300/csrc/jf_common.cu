// Workspace shared by every handle kind (allocation and release).
#include <cstring>

#include "jf_internal.h"

namespace jf {

#ifdef JF_DEBUG_BOUNDS
static unsigned long long* g_trace_host = nullptr;
static unsigned long long* g_trace_dev = nullptr;

unsigned long long* debug_trace_dev() {
  if (!g_trace_dev) {
    void* p = nullptr;
    if (cudaHostAlloc(&p, sizeof(unsigned long long) * kTraceWords, cudaHostAllocMapped) != cudaSuccess) return nullptr;
    std::memset(p, 0, sizeof(unsigned long long) * kTraceWords);
    void* d = nullptr;
    if (cudaHostGetDevicePointer(&d, p, 0) != cudaSuccess) return nullptr;
    g_trace_host = static_cast<unsigned long long*>(p);
    g_trace_dev = static_cast<unsigned long long*>(d);
  }
  return g_trace_dev;
}
#endif

jf_status alloc_common(jf_ctx* h) {
  cudaError_t e;
#ifdef JF_DEBUG_BOUNDS
  debug_trace_dev();
#endif
  if ((e = cudaMalloc(&h->flag, sizeof(int))) != cudaSuccess) return cuda_fail(h, e, "workspace: flag");
  if ((e = cudaMemset(h->flag, 0, sizeof(int))) != cudaSuccess) return cuda_fail(h, e, "workspace: flag");
  if ((e = cudaMalloc(&h->dt_buf, sizeof(double))) != cudaSuccess) return cuda_fail(h, e, "workspace: dt");
  if ((e = cudaMemset(h->dt_buf, 0, sizeof(double))) != cudaSuccess) return cuda_fail(h, e, "workspace: dt");
  void* red = nullptr;
  if ((e = cudaMalloc(&red, 2 * sizeof(ReduceScratch))) != cudaSuccess) return cuda_fail(h, e, "workspace: reduction");
  if ((e = cudaMemset(red, 0, 2 * sizeof(ReduceScratch))) != cudaSuccess) return cuda_fail(h, e, "workspace: reduction");
  h->red_cfl = static_cast<ReduceScratch*>(red);
  h->red_loss = h->red_cfl + 1;
  if ((e = cudaStreamCreateWithFlags(&h->capture_stream, cudaStreamNonBlocking)) != cudaSuccess)
    return cuda_fail(h, e, "workspace: capture stream");
  return JF_OK;
}

void release_all(jf_ctx* h) {
  for (void*& p : h->stage) { if (p) cudaFree(p); p = nullptr; }
  for (void*& p : h->adj) { if (p) cudaFree(p); p = nullptr; }
  for (void*& p : h->sim_stage) { if (p) cudaFree(p); p = nullptr; }
  if (h->flag) cudaFree(h->flag);
  if (h->dt_buf) cudaFree(h->dt_buf);
  if (h->red_cfl) cudaFree(h->red_cfl);
  if (h->d_sims) cudaFree(h->d_sims);
  if (h->desc_done) cudaEventSynchronize(h->desc_done);
  if (h->desc_pinned) cudaFreeHost(h->desc_pinned);
  if (h->desc_done) cudaEventDestroy(h->desc_done);
  h->desc_pinned = nullptr;
  h->desc_done = nullptr;
  if (h->vjp_desc_done) cudaEventSynchronize(h->vjp_desc_done);
  if (h->vjp_desc_host) cudaFreeHost(h->vjp_desc_host);
  if (h->vjp_desc_dev) cudaFree(h->vjp_desc_dev);
  if (h->vjp_desc_done) cudaEventDestroy(h->vjp_desc_done);
  h->vjp_desc_host = h->vjp_desc_dev = nullptr;
  h->vjp_desc_done = nullptr;
  if (h->rec_store) cudaFree(h->rec_store);
  h->rec_store = nullptr;
  h->rec_cap = h->rec_limit = h->rec_used = 0;
  h->rec_defer = false;
  if (h->d_work) cudaFree(h->d_work);
  if (h->d_dt) cudaFree(h->d_dt);
  if (h->d_red) cudaFree(h->d_red);
  if (h->d_cfl) cudaFree(h->d_cfl);
  if (h->d_chunks) cudaFree(h->d_chunks);
  h->d_cfl = nullptr;
  h->d_chunks = nullptr;
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  for (void*& p : h->pipe_buf) { if (p) cudaFree(p); p = nullptr; }
  if (h->pipe_in) cudaStreamDestroy(h->pipe_in);
  if (h->pipe_out) cudaStreamDestroy(h->pipe_out);
  h->pipe_in = h->pipe_out = nullptr;
  for (cudaEvent_t& ev : h->pipe_ev) { if (ev) cudaEventDestroy(ev); ev = nullptr; }
  h->flag = nullptr; h->dt_buf = nullptr; h->red_cfl = h->red_loss = nullptr;
  h->d_sims = nullptr; h->d_work = nullptr; h->d_dt = nullptr; h->d_red = nullptr; h->capture_stream = nullptr;
}

}  // namespace jf

#ifdef JF_DEBUG_BOUNDS
// Host view of the trace buffer (debug build only; not declared in jf.h).
extern "C" unsigned long long* jf_debug_trace_host(void) {
  jf::debug_trace_dev();
  return jf::g_trace_host;
}
#endif

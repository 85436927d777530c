// Workspace shared by every handle kind (allocation and release).
#include "jf_internal.h"

namespace jf {

jf_status alloc_common(jf_ctx* h) {
  cudaError_t e;
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
  if (h->d_work) cudaFree(h->d_work);
  if (h->d_dt) cudaFree(h->d_dt);
  if (h->d_red) cudaFree(h->d_red);
  if (h->d_cfl) cudaFree(h->d_cfl);
  if (h->d_chunks) cudaFree(h->d_chunks);
  h->d_cfl = nullptr;
  h->d_chunks = nullptr;
  if (h->capture_stream) cudaStreamDestroy(h->capture_stream);
  h->flag = nullptr; h->dt_buf = nullptr; h->red_cfl = h->red_loss = nullptr;
  h->d_sims = nullptr; h->d_work = nullptr; h->d_dt = nullptr; h->d_red = nullptr; h->capture_stream = nullptr;
}

}  // namespace jf

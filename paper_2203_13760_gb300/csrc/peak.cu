// FMA-throughput microbenchmark (jf_fma_peak): the ALU roofline of the stage
// kernels is the FP32 (or FP64) fused-multiply-add rate, which the driver's
// measured peaks (a copy bandwidth and a bf16 GEMM rate) do not give.  Every
// thread runs eight independent FMA chains (enough independent work per warp
// to fill the pipes at full occupancy) on values that stay bounded
// (x <- a x + b with 0 < a < 1 converges to b / (1 - a)).
#include "jf_internal.h"

namespace jf {

constexpr int kPeakThreads = 256, kPeakChains = 8, kPeakUnroll = 16;

template <typename T>
__global__ void __launch_bounds__(kPeakThreads) fma_peak_kernel(T a, T b, int iters, T* sink) {
  T x[kPeakChains];
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) x[k] = T(threadIdx.x + k) * T(1e-3);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kPeakUnroll; ++u)
#pragma unroll
      for (int k = 0; k < kPeakChains; ++k) x[k] = fma(x[k], a, b);
  }
  T s = T(0);
#pragma unroll
  for (int k = 0; k < kPeakChains; ++k) s += x[k];
  if (s == T(-1)) *sink = s;  // never true (every x stays positive); keeps the chains live
}

template <typename T>
jf_status fma_peak(int iters, double* flops_per_s, cudaStream_t s) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_peak_kernel<T>, kPeakThreads, 0);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "jf_fma_peak: device query");
  T* sink = nullptr;
  if ((e = cudaMalloc(&sink, sizeof(T))) != cudaSuccess) return cuda_fail(nullptr, e, "jf_fma_peak: cudaMalloc");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int blocks = sms * (per_sm > 0 ? per_sm : 1);
  const T a = T(0.999), b = T(1e-3);
  float ms = 0.0f;
  if (e == cudaSuccess) {
    fma_peak_kernel<T><<<blocks, kPeakThreads, 0, s>>>(a, b, iters / 4 + 1, sink);  // warm-up
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  if (e == cudaSuccess) {
    fma_peak_kernel<T><<<blocks, kPeakThreads, 0, s>>>(a, b, iters, sink);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "jf_fma_peak: launch");
  const double flops = 2.0 * kPeakChains * kPeakUnroll * (double)iters * blocks * kPeakThreads;
  *flops_per_s = ms > 0.0f ? flops / (ms * 1e-3) : 0.0;
  return JF_OK;
}

}  // namespace jf

using namespace jf;

extern "C" jf_status jf_fma_peak(int dtype, int iters, double* flops_per_s, void* stream) {
  if (!flops_per_s || iters < 1 || (dtype != JF_F32 && dtype != JF_F64)) {
    set_error(nullptr, "jf_fma_peak: need dtype JF_F32 or JF_F64, iters >= 1 and an output pointer");
    return JF_ERR_ARG;
  }
  return dtype == JF_F32 ? fma_peak<float>(iters, flops_per_s, (cudaStream_t)stream)
                         : fma_peak<double>(iters, flops_per_s, (cudaStream_t)stream);
}

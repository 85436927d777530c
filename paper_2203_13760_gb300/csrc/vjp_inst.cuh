// Launch wrappers of the stage VJP kernel (one box shape per dimensionality
// and precision).
#pragma once
#include "vjp.cuh"

namespace jf {

template <typename T>
using VjpLaunch = cudaError_t (*)(const VjpArgs<T>& A, const Gas<T>& g, cudaStream_t s);

template <typename T, int DIM, bool VISC, int BX, int BY, int BZ, int MINB>
cudaError_t launch_vjp(const VjpArgs<T>& A, const Gas<T>& g, cudaStream_t s) {
  constexpr size_t smem = vjp_smem_bytes<T, DIM, VISC, BX, BY, BZ>();
  auto k = vjp_stage_kernel<T, DIM, VISC, BX, BY, BZ, MINB>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((A.n[0] + BX - 1) / BX, (A.n[1] + BY - 1) / BY, (A.n[2] + BZ - 1) / BZ);
  k<<<grid, BX * BY * BZ, smem, s>>>(A, g);
  return cudaGetLastError();
}

// Launcher for (dim, visc) in precision T (null if none is compiled).
template <typename T>
VjpLaunch<T> vjp_launcher(int dim, bool visc);

}  // namespace jf

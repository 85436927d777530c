// Launch wrappers of the stage VJP kernels: the box kernel (1D, 2D; one box
// shape per dimensionality and precision) and the z-marching kernel (3D).
#pragma once
#include "vjp.cuh"
#include "vjp3.cuh"

namespace jf {

// scratch: the z-marching kernel's global accumulator ([6][N] elements); the
// box kernel needs none
template <typename T>
using VjpLaunch = cudaError_t (*)(const VjpArgs<T>& A, const Gas<T>& g, T* scratch, cudaStream_t s);

template <typename T, int DIM, bool VISC, int BX, int BY, int BZ, int MINB>
cudaError_t launch_vjp(const VjpArgs<T>& A, const Gas<T>& g, T*, cudaStream_t s) {
  constexpr size_t smem = vjp_smem_bytes<T, DIM, VISC, BX, BY, BZ>();
  auto k = vjp_stage_kernel<T, DIM, VISC, BX, BY, BZ, MINB>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((A.n[0] + BX - 1) / BX, (A.n[1] + BY - 1) / BY, (A.n[2] + BZ - 1) / BZ);
  k<<<grid, BX * BY * BZ, smem, s>>>(A, g);
  return cudaGetLastError();
}

// 3D: clear the accumulator, the z-marching face kernel, the per-cell pass.
// z chunk: about four waves of CTAs (one CTA per SM), 4 .. 32 planes.
template <typename T, bool VISC, int BX, int BY, int NT, int MINB>
cudaError_t launch_vjp3(const VjpArgs<T>& A, const Gas<T>& g, T* Gacc, cudaStream_t s) {
  constexpr size_t smem = vjp3_smem_bytes<T, VISC, BX, BY>();
  auto k = vjp3_kernel<T, VISC, BX, BY, NT, MINB>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 1;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  constexpr int NCW = VISC ? 6 : 5;
  if ((e = cudaMemsetAsync(Gacc, 0, (size_t)NCW * (size_t)A.N * sizeof(T), s)) != cudaSuccess) return e;
  const long long cols = (long long)((A.n[0] + BX - 1) / BX) * ((A.n[1] + BY - 1) / BY);
  long long zc = (A.n[2] * cols + 4LL * sms - 1) / (4LL * sms);
  zc = zc < 4 ? 4 : (zc > 32 ? 32 : zc);
  const int zchunk = (int)zc;
  const dim3 grid((A.n[0] + BX - 1) / BX, (A.n[1] + BY - 1) / BY, (A.n[2] + zchunk - 1) / zchunk);
  k<<<grid, NT, smem, s>>>(A, g, Gacc, zchunk);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  long long blocks = (A.N + 255) / 256;
  if (blocks > 16LL * sms) blocks = 16LL * sms;
  vjp3_finish_kernel<T, VISC><<<(unsigned)blocks, 256, 0, s>>>(A, g, Gacc);
  return cudaGetLastError();
}

// Launcher for (dim, visc) in precision T (null if none is compiled).
template <typename T>
VjpLaunch<T> vjp_launcher(int dim, bool visc);

}  // namespace jf

// Launch wrappers that instantiate the stage kernel for one tile shape.
#pragma once
#include "variants.h"

namespace jf {

template <typename T, int DIM, bool VISC, int BX, int BY>
cudaError_t prepare_stage() {
  constexpr size_t smem = stage_smem_bytes<T, DIM, VISC, BX, BY>();
  return cudaFuncSetAttribute(stage_kernel<T, DIM, VISC, BX, BY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem);
}

template <typename T, int DIM, bool VISC, int BX, int BY>
cudaError_t launch_stage(const StageArgs<T>& A, const Gas<T>& g, cudaStream_t s) {
  constexpr size_t smem = stage_smem_bytes<T, DIM, VISC, BX, BY>();
  const dim3 grid((A.nx + BX - 1) / BX, DIM >= 2 ? (A.ny + BY - 1) / BY : 1,
                  DIM == 3 ? (A.nz + A.zchunk - 1) / A.zchunk : 1);
  stage_kernel<T, DIM, VISC, BX, BY><<<grid, BX * BY, smem, s>>>(A, g);
  return cudaGetLastError();
}

template <typename T, int DIM, bool VISC, int BX, int BY>
StageVariant<T> make_variant() {
  return StageVariant<T>{DIM, VISC, BX, BY, stage_smem_bytes<T, DIM, VISC, BX, BY>(),
                         &prepare_stage<T, DIM, VISC, BX, BY>, &launch_stage<T, DIM, VISC, BX, BY>, nullptr};
}

}  // namespace jf

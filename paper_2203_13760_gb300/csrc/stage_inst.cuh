// Launch wrappers that instantiate the stage kernel for one tile shape.
#pragma once
#include "variants.h"

namespace jf {

// Dynamic shared memory of a launch: the tile buffers, plus the Rusanov-NN
// parameters (at a 16-byte aligned offset) in the kernels of that flux, or the
// per-cell WENO5 face values in the default-scheme kernels.
template <typename T, int DIM, bool VISC, int BX, int BY, int SCH>
constexpr size_t launch_smem() {
  return SCH == SCH_NN ? sizeof(T) * (nn_smem_offset<T, DIM, VISC, BX, BY>() + NN_PARAMS)
                       : stage_smem_bytes<T, DIM, VISC, BX, BY>() +
                             (sch_pc(SCH) ? sizeof(T) * recon_smem_elems<DIM, BX, BY>() : 0);
}

// MINB: CTAs per SM the register allocation must allow (__launch_bounds__).
template <typename T, int DIM, bool VISC, int BX, int BY, int MINB, int SCH>
cudaError_t prepare_stage() {
  constexpr size_t smem = launch_smem<T, DIM, VISC, BX, BY, SCH>();
  return cudaFuncSetAttribute(stage_kernel<T, DIM, VISC, BX, BY, MINB, SCH>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// A.zchunk: planes per CTA of a z-march (DIM_Y2: rows of the 2D grid).
template <typename T, int DIM, bool VISC, int BX, int BY, int MINB, int SCH>
cudaError_t launch_stage(const StageArgs<T>& A0, const Gas<T>& g, cudaStream_t s) {
  const size_t smem = launch_smem<T, DIM, VISC, BX, BY, SCH>();
  StageArgs<T> A = A0;
  if constexpr (DIM == DIM_Y2) rows_as_planes(A);
  const dim3 grid((A.nx + BX - 1) / BX, plane_dims(DIM) == 2 ? (A.ny + BY - 1) / BY : 1,
                  marches(DIM) ? (A.nz + A.zchunk - 1) / A.zchunk : 1);
  stage_kernel<T, DIM, VISC, BX, BY, MINB, SCH><<<grid, Geo<BX, BY, DIM, VISC>::NT, smem, s>>>(A, nullptr, nullptr, 0, 0,
                                                                                          g);
  return cudaGetLastError();
}

template <typename T, int DIM, bool VISC, int BX, int BY, int MINB, int SCH>
cudaError_t prepare_batch(int* blocks_per_sm) {
  auto k = stage_kernel<T, DIM, VISC, BX, BY, MINB, SCH>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)launch_smem<T, DIM, VISC, BX, BY, SCH>());
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, Geo<BX, BY, DIM, VISC>::NT,
                                                       launch_smem<T, DIM, VISC, BX, BY, SCH>());
}

// rows: z-march kernels (3D, DIM_Y2), the planes (rows) of a work item's
// chunk (other kernels ignore it).
template <typename T, int DIM, bool VISC, int BX, int BY, int MINB, int SCH>
cudaError_t launch_batch(const SimDesc<T>* sims, const WorkItem* work, int nwork, int stage, const Gas<T>& g,
                         int* flag, int grid, int rows, cudaStream_t s) {
  const size_t smem = launch_smem<T, DIM, VISC, BX, BY, SCH>();
  StageArgs<T> A{};
  A.flag = flag;
  A.zchunk = rows;
#ifdef JF_DEBUG_BOUNDS
  A.trace = debug_trace_dev();
#endif
  stage_kernel<T, DIM, VISC, BX, BY, MINB, SCH><<<grid, Geo<BX, BY, DIM, VISC>::NT, smem, s>>>(A, sims, work, nwork,
                                                                                          stage, g);
  return cudaGetLastError();
}

template <typename T, int DIM, bool VISC, int BX, int BY, int MINB, int SCH>
StageVariant<T> make_variant() {
  StageVariant<T> v{DIM == DIM_Y2 ? 2 : DIM, VISC, BX, BY, launch_smem<T, DIM, VISC, BX, BY, SCH>(),
                    &prepare_stage<T, DIM, VISC, BX, BY, MINB, SCH>, &launch_stage<T, DIM, VISC, BX, BY, MINB, SCH>,
                    nullptr, nullptr, Geo<BX, BY, DIM, VISC>::NT, SCH, MINB, DIM == DIM_Y2};
  v.prepare_batch = &prepare_batch<T, DIM, VISC, BX, BY, MINB, SCH>;
  v.launch_batch = &launch_batch<T, DIM, VISC, BX, BY, MINB, SCH>;
  return v;
}

}  // namespace jf

// Table of compiled launch variants of the stage kernels (host side).
//
// Each variant is one template instantiation of a tile shape (BX x BY cells
// per CTA) for a dimensionality, precision and physics set.  The host API
// picks the default per configuration; jf_set_variant (the autotuner hook)
// picks another.
#pragma once
#include <cuda_runtime.h>

#include "jf_math.cuh"
#include "stage.cuh"

namespace jf {

template <typename T>
struct StageVariant {
  int dim;
  bool visc;
  int bx, by;
  size_t smem;
  cudaError_t (*prepare)();  // one-time attribute set-up (dynamic shared memory)
  cudaError_t (*launch)(const StageArgs<T>& A, const Gas<T>& g, cudaStream_t s);
  // persistent batched launch over a work list (same tile code)
  cudaError_t (*prepare_batch)(int* blocks_per_sm);
  cudaError_t (*launch_batch)(const SimDesc<T>* sims, const WorkItem* work, int nwork, int stage, const Gas<T>& g,
                              int* flag, int grid, int rows, cudaStream_t s);
  int threads;
  int scheme;    // SCH_DEFAULT, SCH_GENERAL (run-time Table 2 choice), SCH_ROE, SCH_NN or an _EXT form
  int minb;      // CTAs per SM the register allocation was bounded for
  bool ymarch;   // 2D grid, one row of BX cells per tile marching along y (kernel DIM_Y2)
};

// All compiled variants for precision T (defined in stage_f32.cu / stage_f64.cu).
template <typename T>
const StageVariant<T>* stage_variants(int* count);

// The run-time-scheme kernels (SCH_GENERAL), the flux-splitting kernels
// (SCH_ROE), the Rusanov-NN kernels (SCH_NN) and the extended forms of the
// first two (walls, WENO3-JS), in their own translation units
// (stage_*_gen.cu, stage_*_roe.cu, stage_*_nn.cu, stage_*_ext.cu) so that they
// compile in parallel with the default ones.
const StageVariant<float>* general_variants_f32(int* count);
const StageVariant<double>* general_variants_f64(int* count);
const StageVariant<float>* roe_variants_f32(int* count);
const StageVariant<double>* roe_variants_f64(int* count);
const StageVariant<float>* nn_variants_f32(int* count);
const StageVariant<double>* nn_variants_f64(int* count);
const StageVariant<float>* ext_variants_f32(int* count);
const StageVariant<double>* ext_variants_f64(int* count);
// The default-scheme kernels of 2D grids in row tiles marching along y
// (DIM_Y2; stage_*_rows.cu).
const StageVariant<float>* rows_variants_f32(int* count);
const StageVariant<double>* rows_variants_f64(int* count);

}  // namespace jf

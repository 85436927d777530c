// FP32 stage kernels with the scheme chosen at run time (Table 2 variants:
// HLL / Rusanov fluxes, Davis / Toro signal speeds, WENO5-Z), one tile shape
// per dimensionality and physics: 32 x 7 (8 warps, two CTAs per SM at 128
// registers, like the default kernels) with the per-cell reconstruction.
// Compiled with the same approximate division and square root as stage_f32.cu.
#include "stage_inst.cuh"

namespace jf {

const StageVariant<float>* general_variants_f32(int* count) {
  static const StageVariant<float> table[] = {
      make_variant<float, 3, true, 32, 7, 2, SCH_GENERAL>(),
      make_variant<float, 3, false, 32, 7, 2, SCH_GENERAL>(),
      make_variant<float, 2, true, 32, 7, 2, SCH_GENERAL>(),
      make_variant<float, 2, false, 32, 7, 2, SCH_GENERAL>(),
      make_variant<float, 1, true, 128, 1, 2, SCH_GENERAL>(),
      make_variant<float, 1, false, 128, 1, 2, SCH_GENERAL>(),
  };
  *count = (int)(sizeof(table) / sizeof(table[0]));
  return table;
}

}  // namespace jf

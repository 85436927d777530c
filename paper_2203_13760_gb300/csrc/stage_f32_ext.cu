// FP32 stage kernels of the run-time-scheme and ROE families in their
// extended forms: slip walls (mirrored ghost cells) and WENO3-JS on top of
// the Table 2 choices.  The host picks them only for grids with a wall side or
// the WENO3-JS reconstruction, so the plain forms keep their register budget.
// One tile shape per dimensionality and physics.
// Compiled with the same approximate division and square root as stage_f32.cu.
#include "stage_inst.cuh"

namespace jf {

const StageVariant<float>* ext_variants_f32(int* count) {
  static const StageVariant<float> table[] = {
      make_variant<float, 3, true, 32, 8, 2, SCH_GENERAL_EXT>(),
      make_variant<float, 3, false, 32, 8, 2, SCH_GENERAL_EXT>(),
      make_variant<float, 2, true, 32, 8, 2, SCH_GENERAL_EXT>(),
      make_variant<float, 2, false, 32, 8, 2, SCH_GENERAL_EXT>(),
      make_variant<float, 1, true, 128, 1, 2, SCH_GENERAL_EXT>(),
      make_variant<float, 1, false, 128, 1, 2, SCH_GENERAL_EXT>(),
      make_variant<float, 3, true, 32, 7, 2, SCH_ROE_EXT>(),
      make_variant<float, 3, false, 32, 7, 2, SCH_ROE_EXT>(),
      make_variant<float, 2, true, 32, 8, 2, SCH_ROE_EXT>(),
      make_variant<float, 2, false, 32, 8, 2, SCH_ROE_EXT>(),
      make_variant<float, 1, true, 128, 1, 2, SCH_ROE_EXT>(),
      make_variant<float, 1, false, 128, 1, 2, SCH_ROE_EXT>(),
  };
  *count = (int)(sizeof(table) / sizeof(table[0]));
  return table;
}

}  // namespace jf

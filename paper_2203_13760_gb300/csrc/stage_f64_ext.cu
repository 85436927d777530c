// FP64 stage kernels of the run-time-scheme and ROE families in their
// extended forms: slip walls (mirrored ghost cells) and WENO3-JS on top of
// the Table 2 choices.  The host picks them only for grids with a wall side or
// the WENO3-JS reconstruction.  One tile shape per dimensionality and physics.
#include "stage_inst.cuh"

namespace jf {

const StageVariant<double>* ext_variants_f64(int* count) {
  static const StageVariant<double> table[] = {
      make_variant<double, 3, true, 32, 4, 1, SCH_GENERAL_EXT>(),
      make_variant<double, 3, false, 32, 4, 1, SCH_GENERAL_EXT>(),
      make_variant<double, 2, true, 32, 8, 1, SCH_GENERAL_EXT>(),
      make_variant<double, 2, false, 32, 8, 1, SCH_GENERAL_EXT>(),
      make_variant<double, 1, true, 128, 1, 1, SCH_GENERAL_EXT>(),
      make_variant<double, 1, false, 128, 1, 1, SCH_GENERAL_EXT>(),
      make_variant<double, 3, true, 32, 4, 1, SCH_ROE_EXT>(),
      make_variant<double, 3, false, 32, 4, 1, SCH_ROE_EXT>(),
      make_variant<double, 2, true, 32, 8, 1, SCH_ROE_EXT>(),
      make_variant<double, 2, false, 32, 8, 1, SCH_ROE_EXT>(),
      make_variant<double, 1, true, 128, 1, 1, SCH_ROE_EXT>(),
      make_variant<double, 1, false, 128, 1, 1, SCH_ROE_EXT>(),
  };
  *count = (int)(sizeof(table) / sizeof(table[0]));
  return table;
}

}  // namespace jf

// FP64 stage kernels with the scheme chosen at run time (Table 2 variants:
// HLL / Rusanov fluxes, Davis / Toro signal speeds, WENO5-Z), one tile shape
// per dimensionality and physics; in 3D also 32 x 4 beside the default 32 x 6
// (HLL at TGV 128^3: 78.3 against 66.4 M cell-updates/s).
#include "stage_inst.cuh"

namespace jf {

const StageVariant<double>* general_variants_f64(int* count) {
  static const StageVariant<double> table[] = {
      make_variant<double, 3, true, 32, 6, 1, SCH_GENERAL>(),
      make_variant<double, 3, true, 32, 4, 1, SCH_GENERAL>(),
      make_variant<double, 3, false, 32, 6, 1, SCH_GENERAL>(),
      make_variant<double, 3, false, 32, 4, 1, SCH_GENERAL>(),
      make_variant<double, 2, true, 32, 8, 1, SCH_GENERAL>(),
      make_variant<double, 2, false, 32, 8, 1, SCH_GENERAL>(),
      make_variant<double, 1, true, 128, 1, 1, SCH_GENERAL>(),
      make_variant<double, 1, false, 128, 1, 1, SCH_GENERAL>(),
  };
  *count = (int)(sizeof(table) / sizeof(table[0]));
  return table;
}

}  // namespace jf

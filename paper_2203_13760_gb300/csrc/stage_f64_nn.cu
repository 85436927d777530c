// FP64 stage kernels of the Rusanov-NN flux (Section 7.4), reconstruction
// chosen at run time, one tile shape per dimensionality and physics.
#include "stage_inst.cuh"

namespace jf {

const StageVariant<double>* nn_variants_f64(int* count) {
  static const StageVariant<double> table[] = {
      make_variant<double, 3, true, 32, 7, 1, SCH_NN>(),
      make_variant<double, 3, false, 32, 7, 1, SCH_NN>(),
      make_variant<double, 2, true, 32, 7, 1, SCH_NN>(),
      make_variant<double, 2, false, 32, 7, 1, SCH_NN>(),
      make_variant<double, 1, true, 128, 1, 1, SCH_NN>(),
      make_variant<double, 1, false, 128, 1, 1, SCH_NN>(),
  };
  *count = (int)(sizeof(table) / sizeof(table[0]));
  return table;
}

}  // namespace jf

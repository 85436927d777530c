// Instantiations of the stage kernel in FP64.
#include "stage_inst.cuh"

namespace jf {

template <>
const StageVariant<double>* stage_variants<double>(int* count) {
  static const StageVariant<double> table[] = {
      // 3D (the first entry per configuration is the default)
      make_variant<double, 3, true, 16, 8>(),
      make_variant<double, 3, true, 32, 4>(),
      make_variant<double, 3, false, 16, 8>(),
      make_variant<double, 3, false, 32, 4>(),
      // 2D
      make_variant<double, 2, true, 32, 8>(),
      make_variant<double, 2, true, 32, 4>(),
      make_variant<double, 2, false, 32, 8>(),
      make_variant<double, 2, false, 32, 4>(),
      // 1D
      make_variant<double, 1, true, 128, 1>(),
      make_variant<double, 1, false, 128, 1>(),
  };
  *count = (int)(sizeof(table) / sizeof(table[0]));
  return table;
}

}  // namespace jf

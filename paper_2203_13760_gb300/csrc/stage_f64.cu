// Instantiations of the stage kernel in FP64 (IEEE division and square root).
#include "stage_inst.cuh"

namespace jf {

template <>
const StageVariant<double>* stage_variants<double>(int* count) {
  static const StageVariant<double> table[] = {
      // 3D (the first entry per configuration is the default)
      make_variant<double, 3, true, 32, 4, 1>(),
      make_variant<double, 3, true, 32, 2, 2>(),
      make_variant<double, 3, false, 32, 4, 1>(),
      make_variant<double, 3, false, 32, 2, 2>(),
      // 2D
      make_variant<double, 2, true, 32, 8, 1>(),
      make_variant<double, 2, true, 32, 4, 2>(),
      make_variant<double, 2, false, 32, 8, 1>(),
      make_variant<double, 2, false, 32, 4, 2>(),
      // 1D
      make_variant<double, 1, true, 128, 1, 1>(),
      make_variant<double, 1, false, 128, 1, 1>(),
  };
  *count = (int)(sizeof(table) / sizeof(table[0]));
  return table;
}

}  // namespace jf

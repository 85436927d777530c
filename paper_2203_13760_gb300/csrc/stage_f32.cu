// Instantiations of the stage kernel in FP32.
#include "stage_inst.cuh"

namespace jf {

template <>
const StageVariant<float>* stage_variants<float>(int* count) {
  static const StageVariant<float> table[] = {
      // 3D (the first entry per configuration is the default)
      make_variant<float, 3, true, 32, 8>(),
      make_variant<float, 3, true, 32, 4>(),
      make_variant<float, 3, false, 32, 8>(),
      make_variant<float, 3, false, 32, 4>(),
      // 2D
      make_variant<float, 2, true, 32, 8>(),
      make_variant<float, 2, true, 32, 4>(),
      make_variant<float, 2, true, 64, 4>(),
      make_variant<float, 2, false, 32, 8>(),
      make_variant<float, 2, false, 32, 4>(),
      make_variant<float, 2, false, 64, 4>(),
      // 1D
      make_variant<float, 1, true, 128, 1>(),
      make_variant<float, 1, false, 128, 1>(),
  };
  *count = (int)(sizeof(table) / sizeof(table[0]));
  return table;
}

}  // namespace jf

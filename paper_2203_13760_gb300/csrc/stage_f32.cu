// Instantiations of the stage kernel in FP32.  This translation unit is
// compiled with approximate division and square root (-prec-div=false
// -prec-sqrt=false -ftz=true): the FP32 path meets its parity bar with them
// and they cut the instruction count of WENO5 / HLLC substantially.
#include "stage_inst.cuh"

namespace jf {

template <>
const StageVariant<float>* stage_variants<float>(int* count) {
  static const StageVariant<float> table[] = {
      // 3D (the first entry per configuration is the default)
      make_variant<float, 3, true, 32, 8, 2>(),
      make_variant<float, 3, true, 32, 6, 3>(),
      make_variant<float, 3, true, 32, 4, 3>(),
      make_variant<float, 3, false, 32, 8, 2>(),
      make_variant<float, 3, false, 32, 6, 3>(),
      make_variant<float, 3, false, 32, 4, 3>(),
      // 2D
      make_variant<float, 2, true, 32, 8, 2>(),
      make_variant<float, 2, true, 32, 4, 4>(),
      make_variant<float, 2, false, 32, 8, 2>(),
      make_variant<float, 2, false, 32, 4, 4>(),
      // 1D
      make_variant<float, 1, true, 128, 1, 2>(),
      make_variant<float, 1, false, 128, 1, 2>(),
  };
  *count = (int)(sizeof(table) / sizeof(table[0]));
  return table;
}

}  // namespace jf

// FP32 stage kernels of the Rusanov-NN flux (Section 7.4), reconstruction
// chosen at run time.  The network's hidden layers keep 64 values per face
// thread live, so these kernels are bounded for fewer CTAs per SM than the
// other families (no register spills).
// Compiled with the same approximate division and square root as stage_f32.cu.
#include "stage_inst.cuh"

namespace jf {

const StageVariant<float>* nn_variants_f32(int* count) {
  static const StageVariant<float> table[] = {
      make_variant<float, 3, true, 32, 7, 1, SCH_NN>(),
      make_variant<float, 3, false, 32, 7, 1, SCH_NN>(),
      // 2D: 32 x 3 tiles (4 warps, two CTAs per SM: up to 256 registers) fill
      // the SMs on small grids such as the 32^2 grids of a training batch
      make_variant<float, 2, true, 32, 3, 2, SCH_NN>(),
      make_variant<float, 2, true, 32, 8, 1, SCH_NN>(),
      make_variant<float, 2, false, 32, 3, 2, SCH_NN>(),
      make_variant<float, 2, false, 32, 8, 1, SCH_NN>(),
      make_variant<float, 2, false, 32, 7, 1, SCH_NN>(),
      make_variant<float, 1, true, 128, 1, 1, SCH_NN>(),
      make_variant<float, 1, false, 128, 1, 1, SCH_NN>(),
  };
  *count = (int)(sizeof(table) / sizeof(table[0]));
  return table;
}

}  // namespace jf

// FP32 stage kernels of the flux-splitting ROE setup (Section 3.3,
// Flux-Splitting approach; Section 5), in several tile shapes: the larger face
// computation needs more registers than the Godunov kernels, and which
// register / occupancy trade-off wins is measured (jf_set_variant, autotune).
// The first 3D entry is the default.  Measured at TGV 256^3 (viscous, stage
// ms): 32 x 7 at two CTAs per SM (8 warps, 128 registers) 2.43; 32 x 15 at
// one (16 warps, 128 registers) 2.41; 32 x 8 at two (9 warps: 96 registers,
// spilling) 2.87; 32 x 8 at one (168 registers) 2.88.
// Compiled with the same approximate division and square root as stage_f32.cu.
#include "stage_inst.cuh"

namespace jf {

const StageVariant<float>* roe_variants_f32(int* count) {
  static const StageVariant<float> table[] = {
      make_variant<float, 3, true, 32, 7, 2, SCH_ROE>(),
      make_variant<float, 3, true, 32, 15, 1, SCH_ROE>(),
      make_variant<float, 3, true, 32, 8, 2, SCH_ROE>(),
      make_variant<float, 3, true, 32, 8, 1, SCH_ROE>(),
      make_variant<float, 3, true, 32, 4, 2, SCH_ROE>(),
      make_variant<float, 3, true, 32, 4, 3, SCH_ROE>(),
      make_variant<float, 3, false, 32, 7, 2, SCH_ROE>(),
      make_variant<float, 3, false, 32, 15, 1, SCH_ROE>(),
      make_variant<float, 3, false, 32, 8, 2, SCH_ROE>(),
      make_variant<float, 3, false, 32, 8, 1, SCH_ROE>(),
      make_variant<float, 3, false, 32, 4, 2, SCH_ROE>(),
      make_variant<float, 3, false, 32, 4, 3, SCH_ROE>(),
      make_variant<float, 2, true, 32, 8, 2, SCH_ROE>(),
      make_variant<float, 2, true, 32, 4, 3, SCH_ROE>(),
      make_variant<float, 2, false, 32, 8, 2, SCH_ROE>(),
      make_variant<float, 2, false, 32, 4, 3, SCH_ROE>(),
      make_variant<float, 1, true, 128, 1, 2, SCH_ROE>(),
      make_variant<float, 1, false, 128, 1, 2, SCH_ROE>(),
  };
  *count = (int)(sizeof(table) / sizeof(table[0]));
  return table;
}

}  // namespace jf

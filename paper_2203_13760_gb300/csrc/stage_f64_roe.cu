// FP64 stage kernels of the flux-splitting ROE setup (Section 3.3,
// Flux-Splitting approach; Section 5), in several tile shapes: the larger face
// computation needs more registers than the Godunov kernels, and which
// register / occupancy trade-off wins is measured (jf_set_variant, autotune):
// in 3D 32 x 6 at one CTA per SM (TGV 128^3: 41.8 against 34.7 M
// cell-updates/s for 32 x 4).
#include "stage_inst.cuh"

namespace jf {

const StageVariant<double>* roe_variants_f64(int* count) {
  static const StageVariant<double> table[] = {
      make_variant<double, 3, true, 32, 6, 1, SCH_ROE>(),
      make_variant<double, 3, true, 32, 4, 1, SCH_ROE>(),
      make_variant<double, 3, true, 32, 2, 2, SCH_ROE>(),
      make_variant<double, 3, false, 32, 6, 1, SCH_ROE>(),
      make_variant<double, 3, false, 32, 4, 1, SCH_ROE>(),
      make_variant<double, 3, false, 32, 2, 2, SCH_ROE>(),
      make_variant<double, 2, true, 32, 8, 1, SCH_ROE>(),
      make_variant<double, 2, true, 32, 4, 2, SCH_ROE>(),
      make_variant<double, 2, false, 32, 8, 1, SCH_ROE>(),
      make_variant<double, 2, false, 32, 4, 2, SCH_ROE>(),
      make_variant<double, 1, true, 128, 1, 1, SCH_ROE>(),
      make_variant<double, 1, false, 128, 1, 1, SCH_ROE>(),
  };
  *count = (int)(sizeof(table) / sizeof(table[0]));
  return table;
}

}  // namespace jf

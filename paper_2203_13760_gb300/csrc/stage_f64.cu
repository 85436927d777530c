// Instantiations of the stage kernel in FP64 (IEEE division and square root).
#include <vector>

#include "stage_inst.cuh"

namespace jf {

// The default-scheme kernels (WENO5-JS, HLLC, Einfeldt) of every tile shape,
// then the run-time-scheme kernels of stage_f64_gen.cu (one tile shape each)
// and the flux-splitting kernels of stage_f64_roe.cu.
template <>
const StageVariant<double>* stage_variants<double>(int* count) {
  static const std::vector<StageVariant<double>> table = [] {
    std::vector<StageVariant<double>> v = {
      // 3D (the first entry per configuration is the default): 32 x 6, one
      // CTA of 7 warps per SM (208 KB of shared memory), measured at TGV 256^3
      // 82.2 M cell-updates/s against 68.8 M for 32 x 4 (5 warps) and 49.1 M
      // for 32 x 2 at two CTAs per SM
      make_variant<double, 3, true, 32, 6, 1, SCH_DEFAULT>(),
      make_variant<double, 3, true, 32, 4, 1, SCH_DEFAULT>(),
      make_variant<double, 3, true, 32, 2, 2, SCH_DEFAULT>(),
      make_variant<double, 3, false, 32, 6, 1, SCH_DEFAULT>(),
      make_variant<double, 3, false, 32, 4, 1, SCH_DEFAULT>(),
      make_variant<double, 3, false, 32, 2, 2, SCH_DEFAULT>(),
      // 2D
      make_variant<double, 2, true, 32, 8, 1, SCH_DEFAULT>(),
      make_variant<double, 2, true, 32, 4, 2, SCH_DEFAULT>(),
      make_variant<double, 2, false, 32, 8, 1, SCH_DEFAULT>(),
      make_variant<double, 2, false, 32, 4, 2, SCH_DEFAULT>(),
      // 1D
      make_variant<double, 1, true, 128, 1, 1, SCH_DEFAULT>(),
      make_variant<double, 1, false, 128, 1, 1, SCH_DEFAULT>(),
    };
    int ng = 0;
    const StageVariant<double>* gen = general_variants_f64(&ng);
    v.insert(v.end(), gen, gen + ng);
    const StageVariant<double>* roe = roe_variants_f64(&ng);
    v.insert(v.end(), roe, roe + ng);
    const StageVariant<double>* nn = nn_variants_f64(&ng);
    v.insert(v.end(), nn, nn + ng);
    const StageVariant<double>* ext = ext_variants_f64(&ng);
    v.insert(v.end(), ext, ext + ng);
    const StageVariant<double>* rows = rows_variants_f64(&ng);
    v.insert(v.end(), rows, rows + ng);
    return v;
  }();
  *count = (int)table.size();
  return table.data();
}

}  // namespace jf

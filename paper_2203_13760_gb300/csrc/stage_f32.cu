// Instantiations of the stage kernel in FP32.  This translation unit is
// compiled with approximate division and square root (-prec-div=false
// -prec-sqrt=false -ftz=true): the FP32 path meets its parity bar with them
// and they cut the instruction count of WENO5 / HLLC substantially.
#include <vector>

#include "stage_inst.cuh"

namespace jf {

// The default-scheme kernels (WENO5-JS, HLLC, Einfeldt) of every tile shape,
// then the run-time-scheme kernels of stage_f32_gen.cu (one tile shape each)
// and the flux-splitting kernels of stage_f32_roe.cu.
// 3D default tile: 32 x 7 cells, 8 warps (seven face/cell rows and the warp
// of the extra faces), two CTAs per SM.  Registers are allocated to warps in
// groups of four, so two 9-warp CTAs (32 x 8) count as 20 warps and cap a
// thread at 96 registers (the kernel then spills); two 8-warp CTAs allow
// 128.  Measured at TGV 256^3: 32 x 7 1.64 ms, 32 x 8 1.75 ms, 32 x 15 (one
// CTA per SM) 1.77 ms.  In 2D, 32 x 7 is also the default (Kelvin-Helmholtz
// 2048^2 stage: 0.254 ms vs 0.264 ms for 32 x 8; batches: equal).
template <>
const StageVariant<float>* stage_variants<float>(int* count) {
  static const std::vector<StageVariant<float>> table = [] {
    std::vector<StageVariant<float>> v = {
      // 3D (the first entry per configuration is the default)
      make_variant<float, 3, true, 32, 7, 2, SCH_DEFAULT>(),
      make_variant<float, 3, true, 32, 8, 2, SCH_DEFAULT>(),
      make_variant<float, 3, true, 32, 15, 1, SCH_DEFAULT>(),
      make_variant<float, 3, true, 32, 6, 3, SCH_DEFAULT>(),
      make_variant<float, 3, true, 32, 4, 3, SCH_DEFAULT>(),
      make_variant<float, 3, false, 32, 7, 2, SCH_DEFAULT>(),
      make_variant<float, 3, false, 32, 8, 2, SCH_DEFAULT>(),
      make_variant<float, 3, false, 32, 15, 1, SCH_DEFAULT>(),
      make_variant<float, 3, false, 32, 6, 3, SCH_DEFAULT>(),
      make_variant<float, 3, false, 32, 4, 3, SCH_DEFAULT>(),
      // 2D
      make_variant<float, 2, true, 32, 7, 2, SCH_DEFAULT>(),
      make_variant<float, 2, true, 32, 8, 2, SCH_DEFAULT>(),
      make_variant<float, 2, true, 32, 4, 4, SCH_DEFAULT>(),
      make_variant<float, 2, false, 32, 7, 2, SCH_DEFAULT>(),
      make_variant<float, 2, false, 32, 8, 2, SCH_DEFAULT>(),
      make_variant<float, 2, false, 32, 4, 4, SCH_DEFAULT>(),
      // 1D
      make_variant<float, 1, true, 128, 1, 2, SCH_DEFAULT>(),
      make_variant<float, 1, false, 128, 1, 2, SCH_DEFAULT>(),
    };
    int ng = 0;
    const StageVariant<float>* gen = general_variants_f32(&ng);
    v.insert(v.end(), gen, gen + ng);
    const StageVariant<float>* roe = roe_variants_f32(&ng);
    v.insert(v.end(), roe, roe + ng);
    const StageVariant<float>* nn = nn_variants_f32(&ng);
    v.insert(v.end(), nn, nn + ng);
    const StageVariant<float>* ext = ext_variants_f32(&ng);
    v.insert(v.end(), ext, ext + ng);
    const StageVariant<float>* rows = rows_variants_f32(&ng);
    v.insert(v.end(), rows, rows + ng);
    return v;
  }();
  *count = (int)table.size();
  return table.data();
}

}  // namespace jf

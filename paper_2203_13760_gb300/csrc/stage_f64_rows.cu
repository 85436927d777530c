// FP64 stage kernels of 2D grids in row tiles marching along y (the FP32
// forms are in stage_f32_rows.cu): one row of 128 cells per CTA, the default
// scheme and the run-time Godunov schemes.
#include "stage_inst.cuh"

namespace jf {

const StageVariant<double>* rows_variants_f64(int* count) {
  static const StageVariant<double> table[] = {
      make_variant<double, DIM_Y2, true, 128, 1, 2, SCH_DEFAULT>(),
      make_variant<double, DIM_Y2, false, 128, 1, 2, SCH_DEFAULT>(),
      make_variant<double, DIM_Y2, true, 128, 1, 2, SCH_GENERAL>(),
      make_variant<double, DIM_Y2, false, 128, 1, 2, SCH_GENERAL>(),
  };
  *count = (int)(sizeof(table) / sizeof(table[0]));
  return table;
}

}  // namespace jf

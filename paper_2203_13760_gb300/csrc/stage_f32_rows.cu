// FP32 default-scheme stage kernels (WENO5-JS, HLLC, Einfeldt) of 2D grids in
// row tiles: a CTA holds one row of BX cells (BX + 32 threads) and marches
// along y over a chunk of rows with the six-slot ring of the 3D kernel, so
// that every row of the grid is loaded and reconstructed along y about once
// (the 32 x 7 tiles of the 2D kernel load 2.2 cells and reconstruct 9/7
// cells along y per cell).  Row widths 128, 224 and 96 cells at three, two
// and four CTAs per SM (16 or 15 warps per SM).
// Compiled with the same approximate division and square root as stage_f32.cu.
#include "stage_inst.cuh"

namespace jf {

const StageVariant<float>* rows_variants_f32(int* count) {
  static const StageVariant<float> table[] = {
      make_variant<float, DIM_Y2, true, 128, 1, 3, SCH_DEFAULT>(),
      make_variant<float, DIM_Y2, true, 224, 1, 2, SCH_DEFAULT>(),
      make_variant<float, DIM_Y2, true, 96, 1, 4, SCH_DEFAULT>(),
      make_variant<float, DIM_Y2, false, 128, 1, 3, SCH_DEFAULT>(),
      make_variant<float, DIM_Y2, false, 224, 1, 2, SCH_DEFAULT>(),
      make_variant<float, DIM_Y2, false, 96, 1, 4, SCH_DEFAULT>(),
      // the run-time Godunov schemes (Table 2 variants), 128 cells per row
      make_variant<float, DIM_Y2, true, 128, 1, 3, SCH_GENERAL>(),
      make_variant<float, DIM_Y2, false, 128, 1, 3, SCH_GENERAL>(),
  };
  *count = (int)(sizeof(table) / sizeof(table[0]));
  return table;
}

}  // namespace jf

// Instantiations of the stage VJP kernel in FP32 (approximate division and
// square root, like the forward FP32 kernels).
#include "vjp_inst.cuh"

namespace jf {

template <>
VjpLaunch<float> vjp_launcher<float>(int dim, bool visc) {
  if (dim == 3) return visc ? &launch_vjp<float, 3, true, 8, 8, 8, 1> : &launch_vjp<float, 3, false, 8, 8, 8, 1>;
  if (dim == 2) return visc ? &launch_vjp<float, 2, true, 16, 16, 1, 2> : &launch_vjp<float, 2, false, 16, 16, 1, 2>;
  if (dim == 1) return visc ? &launch_vjp<float, 1, true, 128, 1, 1, 2> : &launch_vjp<float, 1, false, 128, 1, 1, 2>;
  return nullptr;
}

}  // namespace jf

// Instantiations of the stage VJP kernels in FP32 (approximate division and
// square root, like the forward FP32 kernels): 3D marches along z over
// 32 x 8 columns (512 threads, one CTA per SM by shared memory).
#include "vjp_inst.cuh"

namespace jf {

template <>
VjpLaunch<float> vjp_launcher<float>(int dim, bool visc) {
  if (dim == 3) return visc ? &launch_vjp3<float, true, 32, 8, 512, 1> : &launch_vjp3<float, false, 32, 8, 512, 1>;
  if (dim == 2) return visc ? &launch_vjp<float, 2, true, 16, 16, 1, 2> : &launch_vjp<float, 2, false, 16, 16, 1, 2>;
  if (dim == 1) return visc ? &launch_vjp<float, 1, true, 128, 1, 1, 2> : &launch_vjp<float, 1, false, 128, 1, 1, 2>;
  return nullptr;
}

}  // namespace jf

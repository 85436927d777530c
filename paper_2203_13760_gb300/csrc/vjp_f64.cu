// Instantiations of the stage VJP kernels in FP64: 3D marches along z over
// 16 x 8 columns (256 threads), 16 x 4 (128 threads) with viscous fluxes,
// whose cotangent rings of the tangential derivatives need the room; the FP64
// plane rings fill the shared memory of one CTA per SM.
#include "vjp_inst.cuh"

namespace jf {

template <>
VjpLaunch<double> vjp_launcher<double>(int dim, bool visc) {
  if (dim == 3) return visc ? &launch_vjp3<double, true, 16, 4, 128, 1> : &launch_vjp3<double, false, 16, 8, 256, 1>;
  if (dim == 2)
    return visc ? &launch_vjp<double, 2, true, 16, 16, 1, 2> : &launch_vjp<double, 2, false, 16, 16, 1, 2>;
  if (dim == 1) return visc ? &launch_vjp<double, 1, true, 128, 1, 1, 2> : &launch_vjp<double, 1, false, 128, 1, 1, 2>;
  return nullptr;
}

}  // namespace jf

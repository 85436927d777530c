// Instantiations of the stage VJP kernel in FP64 (3D boxes of 4^3 cells so
// that the 5-cell halo of FP64 primitives fits in shared memory).
#include "vjp_inst.cuh"

namespace jf {

template <>
VjpLaunch<double> vjp_launcher<double>(int dim, bool visc) {
  if (dim == 3) return visc ? &launch_vjp<double, 3, true, 4, 4, 4, 1> : &launch_vjp<double, 3, false, 4, 4, 4, 1>;
  if (dim == 2)
    return visc ? &launch_vjp<double, 2, true, 16, 16, 1, 2> : &launch_vjp<double, 2, false, 16, 16, 1, 2>;
  if (dim == 1) return visc ? &launch_vjp<double, 1, true, 128, 1, 1, 2> : &launch_vjp<double, 1, false, 128, 1, 1, 2>;
  return nullptr;
}

}  // namespace jf

// Instantiations of the stage VJP kernel in FP64.
#include "vjp_inst.cuh"

namespace jf {

template <>
VjpLaunch<double> vjp_launcher<double>(int dim, bool visc) {
  if (dim == 2) return visc ? &launch_vjp<double, 2, true, 16, 16> : &launch_vjp<double, 2, false, 16, 16>;
  if (dim == 1) return visc ? &launch_vjp<double, 1, true, 128, 1> : &launch_vjp<double, 1, false, 128, 1>;
  return nullptr;
}

}  // namespace jf

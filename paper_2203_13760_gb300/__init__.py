"""GB300 (sm_103a) implementation of the finite-volume RK3 stage of the
compressible Euler / Navier-Stokes equations of JAX-FLUIDS (arXiv 2203.13760).

Modules:
  jf        ctypes binding of libjf.so (include/jf.h): Solver, Batch
  autograd  torch.autograd.Function of the RK3 step and checkpointed rollouts
  autotune  variant sweep (tile shape, z chunk) cached to JSON
  inputs    seeded synthetic initial states shaped like the paper's cases
Submodules are imported lazily so that ``inputs`` needs neither torch nor CUDA.
"""
__all__ = ["jf", "autograd", "autotune", "inputs"]

// Host emulation of the stage kernel: the kernel source of stage.cuh (a copy
// whose dynamic shared-memory declaration points at emu_smem()) compiled for
// the CPU with the stand-ins of cuda_stub/cuda_runtime.h.  Each CTA of the
// launch grid runs in turn as Geo::NT std::threads sharing one std::barrier;
// its shared memory and every global array are heap buffers of exactly their
// size (filled with NaN bit patterns), so that AddressSanitizer reports any
// access outside them and the oracle comparison shows any read of a slot the
// kernel did not write.  Test infrastructure only (tests/test_host_emulation.py).
#include <cstring>
#include <memory>
#include <thread>
#include <vector>

#include "stage.cuh"

thread_local uint3 threadIdx;
thread_local uint3 blockIdx;
dim3 blockDim, gridDim;
static std::barrier<>* g_bar = nullptr;
static unsigned char* g_smem = nullptr;
void emu_syncthreads() { g_bar->arrive_and_wait(); }
unsigned char* emu_smem() { return g_smem; }

using namespace jf;

template <typename T, int DIM, bool VISC, int BX, int BY>
static void run(StageArgs<T> A, const Gas<T>& g) {
  using G = Geo<BX, BY, DIM, VISC>;
  if constexpr (DIM == DIM_Y2) rows_as_planes(A);
  const size_t smem = sizeof(T) * (stage_smem_elems<T, DIM, VISC, BX, BY>() + recon_smem_elems<DIM, BX, BY>());
  gridDim.x = (A.nx + BX - 1) / BX;
  gridDim.y = plane_dims(DIM) == 2 ? (A.ny + BY - 1) / BY : 1;
  gridDim.z = marches(DIM) ? (A.nz + A.zchunk - 1) / A.zchunk : 1;
  blockDim.x = G::NT;
  for (unsigned bz = 0; bz < gridDim.z; ++bz)
    for (unsigned by = 0; by < gridDim.y; ++by)
      for (unsigned bx = 0; bx < gridDim.x; ++bx) {
        std::unique_ptr<unsigned char[]> sm(new unsigned char[smem]);
        std::memset(sm.get(), 0xFF, smem);
        g_smem = sm.get();
        std::barrier<> bar(G::NT);
        g_bar = &bar;
        std::vector<std::thread> th;
        for (int t = 0; t < G::NT; ++t)
          th.emplace_back([&, t] {
            threadIdx = uint3{(unsigned)t, 0, 0};
            blockIdx = uint3{bx, by, bz};
            stage_kernel<T, DIM, VISC, BX, BY, 1, SCH_DEFAULT>(A, nullptr, nullptr, 0, 0, g);
          });
        for (auto& x : th) x.join();
      }
}

// Kernels: 0 the 2D tiles (FP32 32 x 7, FP64 32 x 8), 1 the 128-wide row
// tiles, 2 the 96-wide and 3 the 224-wide row tiles (FP32), 4 the 3D tiles
// (FP32 32 x 7, FP64 32 x 4).
template <typename T>
static int emulate(int kernel, bool visc, StageArgs<T>& A, const Gas<T>& g) {
  constexpr bool f32 = sizeof(T) == 4;
  switch (kernel) {
    case 0:
      if (visc) run<T, 2, true, 32, f32 ? 7 : 8>(A, g); else run<T, 2, false, 32, f32 ? 7 : 8>(A, g);
      return 0;
    case 1:
      if (visc) run<T, DIM_Y2, true, 128, 1>(A, g); else run<T, DIM_Y2, false, 128, 1>(A, g);
      return 0;
    case 2:
      if (visc) run<T, DIM_Y2, true, 96, 1>(A, g); else run<T, DIM_Y2, false, 96, 1>(A, g);
      return 0;
    case 3:
      if (visc) run<T, DIM_Y2, true, 224, 1>(A, g); else run<T, DIM_Y2, false, 224, 1>(A, g);
      return 0;
    case 4:
      if (visc) run<T, 3, true, 32, f32 ? 7 : 4>(A, g); else run<T, 3, false, 32, f32 ? 7 : 4>(A, g);
      return 0;
  }
  return -1;
}

// One launch: out = L(Us) (rhs_only) or out = a Un + b (Us + dt L(Us)) (Un may
// be null: a = 0).  gas = {gamma, R, mu, lambda, eps}.  Returns the device
// flag (bit 0: non-physical state), or -1 for an unknown kernel.
template <typename T>
static int stage(int kernel, const int* n, const int* periodic, const double* inv_h, const double* gas, int zchunk,
                 int rhs_only, double a, double b, double dt, const T* Us, const T* Un, T* out) {
  const long long N = (long long)n[0] * n[1] * n[2];
  std::unique_ptr<T[]> us(new T[5 * N]), un(Un ? new T[5 * N] : nullptr), o(new T[5 * N]);
  std::memcpy(us.get(), Us, sizeof(T) * 5 * N);
  if (Un) std::memcpy(un.get(), Un, sizeof(T) * 5 * N);
  std::unique_ptr<double[]> dtp(new double[1]);
  dtp[0] = dt;
  int flag = 0;
  StageArgs<T> A;
  std::memset(&A, 0, sizeof A);
  A.Us = us.get();
  A.Un = un.get();
  A.out = o.get();
  A.dt = rhs_only ? nullptr : dtp.get();
  A.nx = n[0];
  A.ny = n[1];
  A.nz = n[2];
  A.N = N;
  for (int d = 0; d < 3; ++d) {
    A.periodic[d] = periodic[d];
    A.inv_h[d] = (T)inv_h[d];
  }
  A.rhs_only = rhs_only;
  A.a = (T)a;
  A.b = (T)b;
  A.zchunk = zchunk;
  A.flag = &flag;
  Gas<T> g;
  std::memset(&g, 0, sizeof g);
  g.gamma = (T)gas[0];
  g.gm1 = (T)(gas[0] - 1.0);
  g.inv_gm1 = (T)(1.0 / (gas[0] - 1.0));
  g.inv_R = (T)(1.0 / gas[1]);
  g.mu = (T)gas[2];
  g.lambda = (T)gas[3];
  g.eps = (T)gas[4];
  if (emulate<T>(kernel, gas[2] > 0.0, A, g) != 0) return -1;
  std::memcpy(out, o.get(), sizeof(T) * 5 * N);
  return flag;
}

extern "C" int emu_stage_f64(int kernel, const int* n, const int* periodic, const double* inv_h, const double* gas,
                             int zchunk, int rhs_only, double a, double b, double dt, const double* Us,
                             const double* Un, double* out) {
  return stage<double>(kernel, n, periodic, inv_h, gas, zchunk, rhs_only, a, b, dt, Us, Un, out);
}

extern "C" int emu_stage_f32(int kernel, const int* n, const int* periodic, const double* inv_h, const double* gas,
                             int zchunk, int rhs_only, double a, double b, double dt, const float* Us,
                             const float* Un, float* out) {
  return stage<float>(kernel, n, periodic, inv_h, gas, zchunk, rhs_only, a, b, dt, Us, Un, out);
}

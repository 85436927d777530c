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

template <typename T, int DIM, bool VISC, int BX, int BY, int SCH = SCH_DEFAULT>
static void run(StageArgs<T> A, const Gas<T>& g) {
  using G = Geo<BX, BY, DIM, VISC>;
  if constexpr (DIM == DIM_Y2) rows_as_planes(A);
  const size_t smem = sizeof(T) * (stage_smem_elems<T, DIM, VISC, BX, BY>() +
                                    (sch_pc(SCH) ? recon_smem_elems<DIM, BX, BY>() : 0));
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
            stage_kernel<T, DIM, VISC, BX, BY, 1, SCH>(A, nullptr, nullptr, 0, 0, g);
          });
        for (auto& x : th) x.join();
      }
}

// The persistent batch form of the same kernel: `ctas` CTAs, in turn, each
// looping over the work items item = blockIdx.x, blockIdx.x + ctas, ...
template <typename T, int DIM, bool VISC, int BX, int BY>
static void run_batch(const StageArgs<T>& A0, const SimDesc<T>* sims, const WorkItem* work, int nwork, int stage,
                      const Gas<T>& g, int ctas) {
  using G = Geo<BX, BY, DIM, VISC>;
  const size_t smem = sizeof(T) * (stage_smem_elems<T, DIM, VISC, BX, BY>() + recon_smem_elems<DIM, BX, BY>());
  gridDim.x = ctas;
  gridDim.y = gridDim.z = 1;
  blockDim.x = G::NT;
  for (int b = 0; b < ctas; ++b) {
    std::unique_ptr<unsigned char[]> sm(new unsigned char[smem]);
    std::memset(sm.get(), 0xFF, smem);
    g_smem = sm.get();
    std::barrier<> bar(G::NT);
    g_bar = &bar;
    std::vector<std::thread> th;
    for (int t = 0; t < G::NT; ++t)
      th.emplace_back([&, t] {
        threadIdx = uint3{(unsigned)t, 0, 0};
        blockIdx = uint3{(unsigned)b, 0, 0};
        stage_kernel<T, DIM, VISC, BX, BY, 1, SCH_DEFAULT>(A0, sims, work, nwork, stage, g);
      });
    for (auto& x : th) x.join();
  }
}

// Kernels: 0 the 2D tiles (FP32 32 x 7, FP64 32 x 8), 1 the 128-wide row
// tiles, 2 the 96-wide and 3 the 224-wide row tiles (FP32), 4 the 3D tiles
// (FP32 32 x 7, FP64 32 x 6); 5 and 6 the run-time-scheme kernels (Table 2
// Godunov variants) of 2D and 3D grids with those tiles, 7 their 128-wide row
// tiles.
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
      if (visc) run<T, 3, true, 32, f32 ? 7 : 6>(A, g); else run<T, 3, false, 32, f32 ? 7 : 6>(A, g);
      return 0;
    case 5:
      if (visc) run<T, 2, true, 32, f32 ? 7 : 8, SCH_GENERAL>(A, g);
      else run<T, 2, false, 32, f32 ? 7 : 8, SCH_GENERAL>(A, g);
      return 0;
    case 6:
      if (visc) run<T, 3, true, 32, f32 ? 7 : 4, SCH_GENERAL>(A, g);
      else run<T, 3, false, 32, f32 ? 7 : 4, SCH_GENERAL>(A, g);
      return 0;
    case 7:
      if (visc) run<T, DIM_Y2, true, 128, 1, SCH_GENERAL>(A, g);
      else run<T, DIM_Y2, false, 128, 1, SCH_GENERAL>(A, g);
      return 0;
  }
  return -1;
}

// One launch: out = L(Us) (rhs_only) or out = a Un + b (Us + dt L(Us)) (Un may
// be null: a = 0).  gas = {gamma, R, mu, lambda, eps, flux, recon, speeds}
// (the last three as the jf_scheme codes).  Returns the device
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
  g.flux = (int)gas[5];
  g.recon = (int)gas[6];
  g.speeds = (int)gas[7];
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

// Stage 1 of a batch (U1 = U + dt L(U) for every simulation) through the
// persistent form: nsim simulations with dims n[3 s + a], periodic flags
// p[3 s + a], spacings 1/h in inv_h[3 s + a] and steps dts[s]; work items as
// the library builds them (tile columns, and for the z-march kernels chunks of
// `rows` planes); `ctas` persistent CTAs.  Us[s] / U1s[s]: 5 N_s values each.
template <typename T>
static int batch_stage1(int kernel, int nsim, const int* n, const int* p, const double* inv_h, const double* gas,
                        int rows, int ctas, const double* dts, const T* const* Us, T* const* U1s) {
  std::vector<std::unique_ptr<T[]>> us, u1;
  std::unique_ptr<double[]> dt(new double[nsim]);
  std::unique_ptr<SimDesc<T>[]> sims(new SimDesc<T>[nsim]);
  std::vector<WorkItem> items;
  const bool f32 = sizeof(T) == 4;
  const int bx = kernel == 0 || kernel == 4 ? 32 : (kernel == 1 ? 128 : (kernel == 2 ? 96 : 224));
  const int by = kernel == 0 ? (f32 ? 7 : 8) : (kernel == 4 ? (f32 ? 7 : 6) : 1);
  for (int s = 0; s < nsim; ++s) {
    const long long N = (long long)n[3 * s] * n[3 * s + 1] * n[3 * s + 2];
    us.emplace_back(new T[5 * N]);
    u1.emplace_back(new T[5 * N]);
    std::memcpy(us.back().get(), Us[s], sizeof(T) * 5 * N);
    dt[s] = dts[s];
    SimDesc<T>& d = sims[s];
    std::memset(&d, 0, sizeof d);
    d.U = us.back().get();
    d.U1 = u1.back().get();
    d.U2 = nullptr;
    d.dt = dt.get() + s;
    d.nx = n[3 * s];
    d.ny = n[3 * s + 1];
    d.nz = n[3 * s + 2];
    d.N = N;
    for (int a = 0; a < 3; ++a) {
      d.periodic[a] = p[3 * s + a];
      d.inv_h[a] = (T)inv_h[3 * s + a];
    }
    const bool rows_kernel = kernel >= 1 && kernel <= 3;
    const int tx = (d.nx + bx - 1) / bx;
    const int ty = rows_kernel ? 1 : (d.ny + by - 1) / by;
    const int marched = rows_kernel ? d.ny : d.nz;
    const int tz = kernel == 0 ? 1 : (marched + rows - 1) / rows;
    for (int z = 0; z < tz; ++z)
      for (int y = 0; y < ty; ++y)
        for (int x = 0; x < tx; ++x) items.push_back(WorkItem{s, x, y, z});
  }
  std::unique_ptr<WorkItem[]> work(new WorkItem[items.size()]);
  std::memcpy(work.get(), items.data(), sizeof(WorkItem) * items.size());
  int flag = 0;
  StageArgs<T> A0;
  std::memset(&A0, 0, sizeof A0);
  A0.flag = &flag;
  A0.zchunk = rows;
  Gas<T> g;
  std::memset(&g, 0, sizeof g);
  g.gamma = (T)gas[0];
  g.gm1 = (T)(gas[0] - 1.0);
  g.inv_gm1 = (T)(1.0 / (gas[0] - 1.0));
  g.inv_R = (T)(1.0 / gas[1]);
  g.mu = (T)gas[2];
  g.lambda = (T)gas[3];
  g.eps = (T)gas[4];
  const bool visc = gas[2] > 0.0;
  const int nw = (int)items.size();
  switch (kernel) {
    case 0:
      if (visc) run_batch<T, 2, true, 32, f32 ? 7 : 8>(A0, sims.get(), work.get(), nw, 1, g, ctas);
      else run_batch<T, 2, false, 32, f32 ? 7 : 8>(A0, sims.get(), work.get(), nw, 1, g, ctas);
      break;
    case 1:
      if (visc) run_batch<T, DIM_Y2, true, 128, 1>(A0, sims.get(), work.get(), nw, 1, g, ctas);
      else run_batch<T, DIM_Y2, false, 128, 1>(A0, sims.get(), work.get(), nw, 1, g, ctas);
      break;
    case 4:
      if (visc) run_batch<T, 3, true, 32, f32 ? 7 : 6>(A0, sims.get(), work.get(), nw, 1, g, ctas);
      else run_batch<T, 3, false, 32, f32 ? 7 : 6>(A0, sims.get(), work.get(), nw, 1, g, ctas);
      break;
    default:
      return -1;
  }
  for (int s = 0; s < nsim; ++s)
    std::memcpy(U1s[s], u1[s].get(), sizeof(T) * 5 * sims[s].N);
  return flag;
}

extern "C" int emu_batch_stage1_f64(int kernel, int nsim, const int* n, const int* p, const double* inv_h,
                                    const double* gas, int rows, int ctas, const double* dts,
                                    const double* const* Us, double* const* U1s) {
  return batch_stage1<double>(kernel, nsim, n, p, inv_h, gas, rows, ctas, dts, Us, U1s);
}

// Host side of the libjf C ABI (include/jf.h): argument checking, workspace
// ownership, launch sequencing of the RK3 step and CUDA-graph capture.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <queue>
#include <vector>

#include "../../include/jf.h"
#include "cfl.cuh"
#include "jf_internal.h"

namespace jf {

static_assert(NN_PARAMS == JF_NN_PARAMS, "network size of the kernels and of the C ABI");

static thread_local std::string g_noctx_error;

void set_error(jf_ctx* h, const std::string& msg) {
  if (h) h->err = msg; else g_noctx_error = msg;
}

jf_status cuda_fail(jf_ctx* h, cudaError_t e, const char* what) {
  char buf[256];
  std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  set_error(h, buf);
  return e == cudaErrorMemoryAllocation ? JF_ERR_OOM : JF_ERR_CUDA;
}

int active_dims(const jf_grid& g) { return g.nz > 1 ? 3 : (g.ny > 1 ? 2 : 1); }

jf_status check_grid(jf_ctx* h, const jf_grid& g) {
  if (g.nx < 1 || g.ny < 1 || g.nz < 1) { set_error(h, "grid: sizes must be >= 1"); return JF_ERR_ARG; }
  if (g.nz > 1 && g.ny == 1) { set_error(h, "grid: active axes must be a prefix (ny == 1 requires nz == 1)"); return JF_ERR_UNSUPPORTED; }
  const int n[3] = {g.nx, g.ny, g.nz};
  for (int d = 0; d < 3; ++d) {
    if (n[d] > 1 && n[d] < 5) { set_error(h, "grid: an active axis needs at least 5 cells"); return JF_ERR_ARG; }
    if (!(g.hi[d] > g.lo[d]) || !std::isfinite(g.hi[d] - g.lo[d])) { set_error(h, "grid: hi must exceed lo"); return JF_ERR_ARG; }
    for (int s = 0; s < 2; ++s)
      if (g.bc[2 * d + s] != JF_BC_PERIODIC && g.bc[2 * d + s] != JF_BC_ZERO_GRADIENT && g.bc[2 * d + s] != JF_BC_WALL) {
        set_error(h, "grid: unknown boundary condition");
        return JF_ERR_ARG;
      }
    if ((g.bc[2 * d] == JF_BC_PERIODIC) != (g.bc[2 * d + 1] == JF_BC_PERIODIC)) {
      set_error(h, "grid: periodic must be set on both sides of an axis");
      return JF_ERR_ARG;
    }
  }
  if ((long long)g.nx * g.ny * g.nz > (1ll << 40)) { set_error(h, "grid: too many cells"); return JF_ERR_ARG; }
  return JF_OK;
}

jf_status check_physics(jf_ctx* h, const jf_gas& gas, const jf_scheme& s) {
  if (!(gas.gamma > 1.0) || !(gas.R > 0.0) || !(gas.mu >= 0.0) || !std::isfinite(gas.mu)) {
    set_error(h, "gas: need gamma > 1, R > 0, mu >= 0");
    return JF_ERR_ARG;
  }
  if ((s.viscous || s.heat) && !(gas.mu > 0.0)) { set_error(h, "scheme: viscous/heat need mu > 0"); return JF_ERR_ARG; }
  if (s.heat && !(gas.Pr > 0.0)) { set_error(h, "gas: heat flux needs Pr > 0"); return JF_ERR_ARG; }
  if (s.dtype != JF_F32 && s.dtype != JF_F64) { set_error(h, "scheme: dtype must be JF_F32 or JF_F64"); return JF_ERR_ARG; }
  if (!(s.weno_eps > 0.0) || !(s.cfl > 0.0)) { set_error(h, "scheme: need weno_eps > 0 and cfl > 0"); return JF_ERR_ARG; }
  if (s.signal_speed < JF_EINFELDT || s.signal_speed > JF_TORO) {
    set_error(h, "scheme: signal_speed must be JF_EINFELDT, JF_DAVIS or JF_TORO");
    return JF_ERR_ARG;
  }
  if (s.flux < JF_FLUX_HLLC || s.flux > JF_FLUX_RUSANOV_NN) {
    set_error(h, "scheme: flux must be JF_FLUX_HLLC, JF_FLUX_HLL, JF_FLUX_RUSANOV, JF_FLUX_ROE or JF_FLUX_RUSANOV_NN");
    return JF_ERR_ARG;
  }
  if (s.recon != JF_WENO5_JS && s.recon != JF_WENO5_Z && s.recon != JF_WENO3_JS) {
    set_error(h, "scheme: recon must be JF_WENO5_JS, JF_WENO5_Z or JF_WENO3_JS");
    return JF_ERR_ARG;
  }
  if (s.integrator < JF_RK3 || s.integrator > JF_EULER) {
    set_error(h, "scheme: integrator must be JF_RK3, JF_RK2 or JF_EULER");
    return JF_ERR_ARG;
  }
  return JF_OK;
}

double spacing(const jf_grid& g, int d) {
  const int n[3] = {g.nx, g.ny, g.nz};
  return (g.hi[d] - g.lo[d]) / n[d];
}

double conductivity(const jf_gas& gas, const jf_scheme& s) {
  return s.heat ? gas.mu * gas.gamma * gas.R / ((gas.gamma - 1.0) * gas.Pr) : 0.0;
}

template <typename T>
Gas<T> make_gas(const jf_gas& gas, const jf_scheme& s) {
  Gas<T> g;
  g.gamma = (T)gas.gamma;
  g.gm1 = (T)(gas.gamma - 1.0);
  g.inv_gm1 = (T)(1.0 / (gas.gamma - 1.0));
  g.inv_R = (T)(1.0 / gas.R);
  g.mu = (T)(s.viscous ? gas.mu : 0.0);
  g.lambda = (T)conductivity(gas, s);
  g.eps = (T)s.weno_eps;
  g.safe = s.safe_recon ? 1 : 0;
  g.flux = s.flux;
  g.recon = s.recon;
  g.speeds = s.signal_speed;
  return g;
}
template Gas<float> make_gas<float>(const jf_gas&, const jf_scheme&);
template Gas<double> make_gas<double>(const jf_gas&, const jf_scheme&);

bool dissipative(const jf_gas& gas, const jf_scheme& s) { return (s.viscous || s.heat) && gas.mu > 0.0; }

CflArgs make_cfl(const jf_grid& g, const jf_gas& gas, const jf_scheme& s) {
  CflArgs a;
  a.N = (long long)g.nx * g.ny * g.nz;
  a.nactive = active_dims(g);
  a.gamma = gas.gamma;
  const double cv = gas.R / (gas.gamma - 1.0);
  const double mu = s.viscous ? gas.mu : 0.0;
  a.kdiff = dissipative(gas, s) ? std::fmax(mu, conductivity(gas, s) / cv) : 0.0;
  double hmin = 1e300;
  for (int d = 0; d < a.nactive; ++d) hmin = std::fmin(hmin, spacing(g, d));
  a.hmin = hmin;
  a.cfl = s.cfl;
  return a;
}

int reduce_blocks(long long N, int sms) {
  long long b = (N + 255) / 256;
  const long long cap = (long long)sms * 8;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

// ------------------------------------------------------------------------
// Variant selection.  A variant = (compiled tile shape, z chunk).  z chunk 0
// (the first, default, one per tile) is chosen from the grid: grids whose
// CTAs fit in one wave of resident CTAs (SMs x the CTAs per SM the tile is
// bounded for) at 32 planes take the planes per CTA that give one wave, so
// that a 32^3 grid does not run on a handful of SMs; larger grids take the
// chunk length in 20..40 whose CTAs, dealt in launch order to the resident
// slots, finish first (schedule_length), which keeps the partly filled last
// wave short.
static const int kZChunks[] = {0, 32, 16, 64, 8};

// Length, in planes, of the greedy schedule of a 3D launch's CTAs: `tiles`
// CTAs per z chunk of z planes (the last chunk shorter), chunk after chunk
// as the hardware issues them, each costing its planes plus kPrologue planes
// for its prologue (six plane loads and a face, measured at about half a
// plane), over `slots` resident CTA slots.
static double schedule_length(long long tiles, int nz, int z, long long slots) {
  constexpr double kPrologue = 0.5;
  std::priority_queue<double, std::vector<double>, std::greater<double>> free_at;
  for (long long i = 0; i < slots; ++i) free_at.push(0.0);
  double end = 0.0;
  for (int z0 = 0; z0 < nz; z0 += z) {
    const double cost = (nz - z0 < z ? nz - z0 : z) + kPrologue;
    for (long long t = 0; t < tiles; ++t) {
      const double done = free_at.top() + cost;
      free_at.pop();
      free_at.push(done);
      end = done > end ? done : end;
    }
  }
  return end;
}

// The rule of jf_auto_zchunk (include/jf.h).
int zchunk_rule(long long nx, long long ny, long long nz, int bx, int by, int ctas_per_sm, int sms) {
  const long long tiles = ((nx + bx - 1) / bx) * ((ny + by - 1) / by);
  const long long slots = (long long)sms * ctas_per_sm;
  long long z = (nz * tiles + slots - 1) / slots;
  if (z < 1) z = 1;
  if (z > 32) {
    z = 32;
    // larger grids: the shortest schedule over 20..40 planes (longest chunk
    // on ties); very large launches keep 32 to bound the host's work
    if (tiles * ((nz + 19) / 20) <= 400000) {
      double best = 0.0;
      for (int c = 40; c >= 20; --c) {
        const double len = schedule_length(tiles, (int)nz, c, slots);
        if (c == 40 || len < best - 1e-9) { best = len; z = c; }
      }
    }
  }
  return (int)z;
}

// ymarch: a 2D grid whose row tiles march along y (chunks of rows).
int auto_zchunk(const jf_ctx* h, int bx, int by, int ctas_per_sm, bool ymarch) {
  const long long key = (((long long)bx * 4096 + by) * 64 + ctas_per_sm) * 2 + (ymarch ? 1 : 0);
  auto it = h->zauto.find(key);
  if (it != h->zauto.end()) return it->second;
  const int cps = ctas_per_sm > 0 ? ctas_per_sm : 1;
  const int z = ymarch ? zchunk_rule(h->grid.nx, 1, h->grid.ny, bx, 1, cps, h->sms)
                       : zchunk_rule(h->grid.nx, h->grid.ny, h->grid.nz, bx, by, cps, h->sms);
  h->zauto[key] = z;
  return z;
}

bool has_walls(const jf_grid& g) {
  for (int i = 0; i < 6; ++i)
    if (g.bc[i] == JF_BC_WALL) return true;
  return false;
}

int scheme_kind(const jf_scheme& s, bool walls) {
  // walls and WENO3-JS need the extended kernel forms
  const bool ext = walls || s.recon == JF_WENO3_JS;
  if (s.flux == JF_FLUX_ROE) return ext ? SCH_ROE_EXT : SCH_ROE;
  if (s.flux == JF_FLUX_RUSANOV_NN) return SCH_NN;
  const bool general = s.flux != JF_FLUX_HLLC || s.signal_speed != JF_EINFELDT || s.recon != JF_WENO5_JS || walls;
  if (!general) return SCH_DEFAULT;
  return ext ? SCH_GENERAL_EXT : SCH_GENERAL;
}

int scheme_kind(const jf_ctx* h) {
  bool walls = h->kind == 0 && has_walls(h->grid);
  for (const jf_grid& g : h->grids) walls = walls || has_walls(g);
  return scheme_kind(h->scheme, walls);
}

template <typename T>
std::vector<std::pair<int, int>> variant_list(int dim, bool visc, int kind) {
  int count = 0;
  const StageVariant<T>* tab = stage_variants<T>(&count);
  std::vector<std::pair<int, int>> out;
  for (int i = 0; i < count; ++i) {
    if (tab[i].dim != dim || tab[i].visc != visc || tab[i].scheme != kind) continue;
    if (dim == 3 || tab[i].ymarch)
      for (int z : kZChunks) out.emplace_back(i, z);
    else
      out.emplace_back(i, 1);
  }
  return out;
}

bool rows_preferred(const jf_grid* grids, int n, int rows_bx, int rows_ctas_per_sm, int tile_bx, int tile_by,
                    int sms) {
  double rows = 0.0, tiles = 0.0, row_tiles = 0.0;
  for (int i = 0; i < n; ++i) {
    const double nx = grids[i].nx, ny = grids[i].ny;
    row_tiles += std::ceil(nx / rows_bx) * ny;
    rows += std::ceil(nx / rows_bx) * rows_bx * ny;
    tiles += std::ceil(nx / tile_bx) * tile_bx * std::ceil(ny / tile_by) * tile_by;
  }
  return rows <= 1.08 * tiles && row_tiles >= 12.0 * sms * (rows_ctas_per_sm > 0 ? rows_ctas_per_sm : 1);
}

template <typename T>
jf_status select_variant(jf_ctx* h, int v, bool prepare) {
  const bool visc = dissipative(h->gas, h->scheme);
  auto list = variant_list<T>(h->dim, visc, scheme_kind(h));
  if (list.empty()) { set_error(h, "no compiled kernel variant for this configuration"); return JF_ERR_UNSUPPORTED; }
  if (v < 0) {  // the first variant, or the first row-tile one (automatic chunk) where rows_preferred says so
    v = 0;
    int count = 0;
    const StageVariant<T>* tab = stage_variants<T>(&count);
    for (int i = 0; i < (int)list.size(); ++i)
      if (tab[list[i].first].ymarch && list[i].second == 0) {
        const StageVariant<T>& r = tab[list[i].first];
        const StageVariant<T>& t0 = tab[list[0].first];
        if (rows_preferred(&h->grid, 1, r.bx, r.minb, t0.bx, t0.by, h->sms)) v = i;
        break;
      }
  }
  if (v >= (int)list.size()) { set_error(h, "variant index out of range"); return JF_ERR_ARG; }
  if (prepare) {
    int count = 0;
    const StageVariant<T>* tab = stage_variants<T>(&count);
    cudaError_t e = tab[list[v].first].prepare();
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaFuncSetAttribute");
  }
  h->variant = v;
  h->table_index = list[v].first;
  h->zchunk = list[v].second;
  return JF_OK;
}

template <typename T>
int describe_variant(jf_ctx* h, int v, char* buf, int len) {
  const bool visc = dissipative(h->gas, h->scheme);
  auto list = variant_list<T>(h->dim, visc, scheme_kind(h));
  if (v < 0 || v >= (int)list.size()) return (int)list.size();
  int count = 0;
  const StageVariant<T>* tab = stage_variants<T>(&count);
  const StageVariant<T>& s = tab[list[v].first];
  if (buf && len > 0) {
    const int z = s.dim == 3 || s.ymarch ? list[v].second : 1;
    const char* march = s.ymarch ? " ymarch" : "";
    if (z == 0)
      std::snprintf(buf, (size_t)len, "tile=%dx%d%s zchunk=auto(%d) smem=%zu ctas/sm=%d", s.bx, s.by, march,
                    auto_zchunk(h, s.bx, s.by, s.minb, s.ymarch), s.smem, s.minb);
    else
      std::snprintf(buf, (size_t)len, "tile=%dx%d%s zchunk=%d smem=%zu ctas/sm=%d", s.bx, s.by, march, z, s.smem,
                    s.minb);
  }
  return (int)list.size();
}

// ------------------------------------------------------------------------
template <typename T>
StageArgs<T> base_args(const jf_ctx* h) {
  StageArgs<T> A;
  std::memset(&A, 0, sizeof A);
  A.nx = h->grid.nx;
  A.ny = h->grid.ny;
  A.nz = h->grid.nz;
  A.N = (long long)A.nx * A.ny * A.nz;
  for (int d = 0; d < 3; ++d) {
    A.periodic[d] = h->grid.bc[2 * d] == JF_BC_PERIODIC;
    A.wall[d] = (h->grid.bc[2 * d] == JF_BC_WALL ? 1 : 0) | (h->grid.bc[2 * d + 1] == JF_BC_WALL ? 2 : 0);
    A.inv_h[d] = (T)(1.0 / spacing(h->grid, d));
  }
  A.zchunk = h->zchunk;
  if (A.zchunk <= 0) {
    int count = 0;
    const StageVariant<T>& v = stage_variants<T>(&count)[h->table_index];
    A.zchunk = auto_zchunk(h, v.bx, v.by, v.minb, v.ymarch);
  }
  A.flag = h->flag;
  return A;
}

template <typename T>
jf_status launch(jf_ctx* h, const StageArgs<T>& A, cudaStream_t s) {
  int count = 0;
  const StageVariant<T>* tab = stage_variants<T>(&count);
  Gas<T> g = make_gas<T>(h->gas, h->scheme);
  if (h->scheme.flux == JF_FLUX_RUSANOV_NN) {
    if (!h->nn) { set_error(h, "Rusanov-NN flux: no network parameters (jf_set_nn)"); return JF_ERR_ARG; }
    g.nn = static_cast<const T*>(h->nn);
  }
  cudaError_t e = tab[h->table_index].launch(A, g, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "stage kernel launch");
  return JF_OK;
}

template <typename T>
jf_status rhs_impl(jf_ctx* h, const void* U, void* dUdt, cudaStream_t s) {
  StageArgs<T> A = base_args<T>(h);
  A.Us = static_cast<const T*>(U);
  A.out = static_cast<T*>(dUdt);
  A.rhs_only = 1;
  A.a = T(0);
  A.b = T(1);
  return launch<T>(h, A, s);
}

template <typename T>
jf_status cfl_impl(jf_ctx* h, const void* U, double* dt_out, double* dt_out2, cudaStream_t s) {
  const CflArgs a = make_cfl(h->grid, h->gas, h->scheme);
  cfl_kernel<T><<<reduce_blocks(a.N, h->sms), 256, 0, s>>>(static_cast<const T*>(U), a, h->red_cfl, dt_out, dt_out2,
                                                            h->flag, nullptr, nullptr, nullptr, nullptr, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "cfl kernel launch");
  return JF_OK;
}

// Per-simulation CFL of a batch (same kernel as the single-grid reduction).
template <typename T>
cudaError_t launch_cfl_batch(const void* sims, const void* chunks, int nchunks, const CflArgs* args,
                             ReduceScratch* red, double* dts, int* flag, cudaStream_t s) {
  CflArgs none{};
  cfl_kernel<T><<<nchunks, 256, 0, s>>>(nullptr, none, nullptr, nullptr, nullptr, flag,
                                        static_cast<const SimDesc<T>*>(sims), static_cast<const CflChunk*>(chunks),
                                        args, red, dts);
  return cudaGetLastError();
}
template cudaError_t launch_cfl_batch<float>(const void*, const void*, int, const CflArgs*, ReduceScratch*, double*,
                                             int*, cudaStream_t);
template cudaError_t launch_cfl_batch<double>(const void*, const void*, int, const CflArgs*, ReduceScratch*, double*,
                                              int*, cudaStream_t);

// One time step of the scheme's integrator: optional CFL reduction, then
// the Shu-Osher stages (TVD-RK3: three; TVD-RK2: two; Euler: one stage into
// U1 and a copy back, since a stage cannot write over its own input).
template <typename T>
jf_status step_impl(jf_ctx* h, void* U, const double* dt_dev, double* dt_used, cudaStream_t s) {
  const double* dt = dt_dev;
  jf_status st;
  if (!dt) {
    st = cfl_impl<T>(h, U, h->dt_buf, dt_used, s);
    if (st != JF_OK) return st;
    dt = h->dt_buf;
  } else if (dt_used && dt_used != dt_dev) {
    cudaError_t e = cudaMemcpyAsync(dt_used, dt_dev, sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpyAsync(dt)");
  }
  T* Un = static_cast<T*>(U);
  T* U1 = static_cast<T*>(h->stage[0]);
  T* U2 = static_cast<T*>(h->stage[1]);
  StageArgs<T> A = base_args<T>(h);
  A.dt = dt;
  // U1 = Un + dt L(Un)
  A.Us = Un; A.Un = nullptr; A.out = U1; A.a = T(0); A.b = T(1);
  if ((st = launch<T>(h, A, s)) != JF_OK) return st;
  if (h->scheme.integrator == JF_EULER) {
    const cudaError_t e = cudaMemcpyAsync(Un, U1, 5 * h->N * sizeof(T), cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? JF_OK : cuda_fail(h, e, "cudaMemcpyAsync(Euler step)");
  }
  if (h->scheme.integrator == JF_RK2) {
    // U^{n+1} = 1/2 Un + 1/2 (U1 + dt L(U1)), written over Un
    A.Us = U1; A.Un = Un; A.out = Un; A.a = T(0.5); A.b = T(0.5);
    return launch<T>(h, A, s);
  }
  // U2 = 3/4 Un + 1/4 (U1 + dt L(U1))
  A.Us = U1; A.Un = Un; A.out = U2; A.a = T(0.75); A.b = T(0.25);
  if ((st = launch<T>(h, A, s)) != JF_OK) return st;
  // U^{n+1} = 1/3 Un + 2/3 (U2 + dt L(U2)), written over Un
  A.Us = U2; A.Un = Un; A.out = Un; A.a = T(1.0 / 3.0); A.b = T(2.0 / 3.0);
  return launch<T>(h, A, s);
}

template <typename T>
jf_status stage_call(jf_ctx* h, const void* Us, const void* Un, void* out, double a, double b, const double* dt,
                     cudaStream_t s) {
  StageArgs<T> A = base_args<T>(h);
  A.Us = static_cast<const T*>(Us);
  A.Un = a != 0.0 ? static_cast<const T*>(Un) : nullptr;
  A.out = static_cast<T*>(out);
  A.a = (T)a;
  A.b = (T)b;
  A.dt = dt;
  return launch<T>(h, A, s);
}

template <typename T>
jf_status loss_impl(jf_ctx* h, const void* U, const void* target, double* loss, void* seed, cudaStream_t s) {
  const long long N = (long long)h->grid.nx * h->grid.ny * h->grid.nz;
  double dV = 1.0;
  for (int d = 0; d < h->dim; ++d) dV *= spacing(h->grid, d);
  loss_density_kernel<T><<<reduce_blocks(N, h->sms), 256, 0, s>>>(
      static_cast<const T*>(U), static_cast<const T*>(target), N, dV, h->red_loss, loss, static_cast<T*>(seed));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "loss kernel launch");
  return JF_OK;
}

template jf_status select_variant<float>(jf_ctx*, int, bool);
template jf_status select_variant<double>(jf_ctx*, int, bool);
template jf_status step_impl<float>(jf_ctx*, void*, const double*, double*, cudaStream_t);
template jf_status step_impl<double>(jf_ctx*, void*, const double*, double*, cudaStream_t);
template jf_status cfl_impl<float>(jf_ctx*, const void*, double*, double*, cudaStream_t);
template jf_status cfl_impl<double>(jf_ctx*, const void*, double*, double*, cudaStream_t);
template StageArgs<float> base_args<float>(const jf_ctx*);
template StageArgs<double> base_args<double>(const jf_ctx*);
template jf_status launch<float>(jf_ctx*, const StageArgs<float>&, cudaStream_t);
template jf_status launch<double>(jf_ctx*, const StageArgs<double>&, cudaStream_t);

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

void free_graphs(jf_ctx* h) {
  for (auto& kv : h->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  h->graphs.clear();
}

}  // namespace jf

using namespace jf;

#define JF_DISPATCH(h, fn, ...) ((h)->scheme.dtype == JF_F32 ? fn<float>(__VA_ARGS__) : fn<double>(__VA_ARGS__))

extern "C" {

const char* jf_version(void) { return "jf 0.1 (sm_103a)"; }

const char* jf_last_error(jf_handle h) { return h ? h->err.c_str() : g_noctx_error.c_str(); }

jf_status jf_init(const jf_grid* grid, const jf_gas* gas, const jf_scheme* scheme, jf_handle* out) {
  if (!grid || !gas || !scheme || !out) { set_error(nullptr, "jf_init: null argument"); return JF_ERR_ARG; }
  *out = nullptr;
  jf_status st;
  if ((st = check_grid(nullptr, *grid)) != JF_OK) return st;
  if ((st = check_physics(nullptr, *gas, *scheme)) != JF_OK) return st;
  jf_ctx* h = new jf_ctx();
  h->kind = 0;
  h->grid = *grid;
  h->gas = *gas;
  h->scheme = *scheme;
  h->dim = active_dims(*grid);
  h->esize = scheme->dtype == JF_F32 ? 4 : 8;
  h->N = (size_t)grid->nx * grid->ny * grid->nz;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e != cudaSuccess) { st = cuda_fail(nullptr, e, "jf_init: device query"); delete h; return st; }
  st = alloc_common(h);
  if (st == JF_OK) {
    const size_t bytes = 5 * h->N * h->esize;
    for (int i = 0; i < 2 && st == JF_OK; ++i) {
      e = cudaMalloc(&h->stage[i], bytes);
      if (e != cudaSuccess) st = cuda_fail(nullptr, e, "jf_init: stage buffer");
    }
  }
  if (st == JF_OK) st = JF_DISPATCH(h, select_variant, h, -1, true);
  if (st != JF_OK) {
    if (!h->err.empty()) set_error(nullptr, h->err);
    jf_destroy(h);
    return st;
  }
  *out = h;
  return JF_OK;
}

jf_status jf_destroy(jf_handle h) {
  if (!h) return JF_OK;
  cudaDeviceSynchronize();
  free_graphs(h);
  release_all(h);
  delete h;
  return JF_OK;
}

jf_status jf_rhs(jf_handle h, const void* U, void* dUdt, void* stream) {
  if (!h || h->kind != 0) { set_error(h, "jf_rhs: not a single-grid handle"); return JF_ERR_ARG; }
  if (!U || !dUdt || !aligned16(U) || !aligned16(dUdt) || U == dUdt) {
    set_error(h, "jf_rhs: U and dUdt must be distinct 16-byte aligned device arrays");
    return JF_ERR_ARG;
  }
  return JF_DISPATCH(h, rhs_impl, h, U, dUdt, (cudaStream_t)stream);
}

jf_status jf_compute_dt(jf_handle h, const void* U, double* dt_dev, void* stream) {
  if (!h || h->kind != 0) { set_error(h, "jf_compute_dt: not a single-grid handle"); return JF_ERR_ARG; }
  if (!U || !dt_dev) { set_error(h, "jf_compute_dt: null pointer"); return JF_ERR_ARG; }
  if (!aligned16(U)) { set_error(h, "jf_compute_dt: U must be a 16-byte aligned device array"); return JF_ERR_ARG; }
  return JF_DISPATCH(h, cfl_impl, h, U, dt_dev, nullptr, (cudaStream_t)stream);
}

jf_status jf_rk3_step(jf_handle h, void* U, const double* dt_dev, double* dt_used_dev, void* stream) {
  if (!h || h->kind != 0) { set_error(h, "jf_rk3_step: not a single-grid handle"); return JF_ERR_ARG; }
  if (!U || !aligned16(U)) { set_error(h, "jf_rk3_step: U must be a 16-byte aligned device array"); return JF_ERR_ARG; }
  return JF_DISPATCH(h, step_impl, h, U, dt_dev, dt_used_dev, (cudaStream_t)stream);
}

// Independent steps of host-resident states, pipelined: state k's upload
// (stream pipe_in), its step (the caller's stream) and its download (stream
// pipe_out) on two device buffers, so that the copies of states k + 1 and
// k - 1 overlap the step of state k.  Events: ev[b] upload of buffer b done,
// ev[2 + b] step on buffer b done, ev[4 + b] download of buffer b done (the
// buffer is free again), ev[6] the caller's stream at entry.
jf_status jf_rk3_step_host(jf_handle h, const void* const* U_in_host, void* const* U_out_host, int n,
                           const double* dt_dev, void* stream) {
  if (!h || h->kind != 0) { set_error(h, "jf_rk3_step_host: not a single-grid handle"); return JF_ERR_ARG; }
  if (n < 0 || (n > 0 && (!U_in_host || !U_out_host))) { set_error(h, "jf_rk3_step_host: bad arguments"); return JF_ERR_ARG; }
  for (int k = 0; k < n; ++k)
    if (!U_in_host[k] || !U_out_host[k]) { set_error(h, "jf_rk3_step_host: null state pointer"); return JF_ERR_ARG; }
  if (n == 0) return JF_OK;
  const size_t bytes = 5 * h->N * h->esize;
  cudaError_t e = cudaSuccess;
  if (!h->pipe_buf[0]) {
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMalloc(&h->pipe_buf[b], bytes);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->pipe_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->pipe_out, cudaStreamNonBlocking);
    for (int i = 0; i < 7 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&h->pipe_ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return cuda_fail(h, e, "jf_rk3_step_host: pipeline set-up");
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t* ev = h->pipe_ev;
  // everything starts after the work already queued on the caller's stream
  e = cudaEventRecord(ev[6], s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->pipe_in, ev[6], 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->pipe_out, ev[6], 0);
  if (e != cudaSuccess) return cuda_fail(h, e, "jf_rk3_step_host: stream ordering");
  for (int k = 0; k < n; ++k) {
    const int b = k & 1;
    void* buf = h->pipe_buf[b];
    // upload once the buffer's previous download has finished
    if (k >= 2) e = cudaStreamWaitEvent(h->pipe_in, ev[4 + b], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(buf, U_in_host[k], bytes, cudaMemcpyHostToDevice, h->pipe_in);
    if (e == cudaSuccess) e = cudaEventRecord(ev[b], h->pipe_in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[b], 0);
    if (e != cudaSuccess) return cuda_fail(h, e, "jf_rk3_step_host: upload");
    jf_status st = JF_DISPATCH(h, step_impl, h, buf, dt_dev, nullptr, s);
    if (st != JF_OK) return st;
    e = cudaEventRecord(ev[2 + b], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->pipe_out, ev[2 + b], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(U_out_host[k], buf, bytes, cudaMemcpyDeviceToHost, h->pipe_out);
    if (e == cudaSuccess) e = cudaEventRecord(ev[4 + b], h->pipe_out);
    if (e != cudaSuccess) return cuda_fail(h, e, "jf_rk3_step_host: download");
  }
  // the caller's stream resumes after the last download
  e = cudaStreamWaitEvent(s, ev[4 + ((n - 1) & 1)], 0);
  if (e == cudaSuccess && n >= 2) e = cudaStreamWaitEvent(s, ev[4 + ((n - 2) & 1)], 0);
  return e == cudaSuccess ? JF_OK : cuda_fail(h, e, "jf_rk3_step_host: join");
}

jf_status jf_stage(jf_handle h, const void* Us, const void* Un, void* out, double a, double b, const double* dt_dev,
                   void* stream) {
  if (!h || h->kind != 0) { set_error(h, "jf_stage: not a single-grid handle"); return JF_ERR_ARG; }
  if (!Us || !out || !dt_dev || !aligned16(Us) || !aligned16(out) || (Un && !aligned16(Un)) || Us == out ||
      (a != 0.0 && !Un)) {
    set_error(h, "jf_stage: bad arguments");
    return JF_ERR_ARG;
  }
  return JF_DISPATCH(h, stage_call, h, Us, Un, out, a, b, dt_dev, (cudaStream_t)stream);
}

jf_status jf_rk3_run(jf_handle h, void* U, int nsteps, const double* dt_dev, double* dt_hist_dev, void* stream) {
  if (!h || h->kind != 0) { set_error(h, "jf_rk3_run: not a single-grid handle"); return JF_ERR_ARG; }
  if (!U || !aligned16(U) || nsteps < 0) { set_error(h, "jf_rk3_run: bad arguments"); return JF_ERR_ARG; }
  if (nsteps == 0) return JF_OK;
  const GraphKey key{U, nsteps, dt_dev, dt_hist_dev, h->variant};
  auto it = h->graphs.find(key);
  if (it == h->graphs.end()) {
    cudaStream_t cs = h->capture_stream;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamBeginCapture");
    jf_status st = JF_OK;
    for (int s = 0; s < nsteps && st == JF_OK; ++s)
      st = JF_DISPATCH(h, step_impl, h, U, dt_dev, dt_hist_dev ? dt_hist_dev + s : nullptr, cs);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cs, &graph);
    if (st != JF_OK) { if (graph) cudaGraphDestroy(graph); return st; }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(h, e, "cudaGraphInstantiate"); }
    it = h->graphs.emplace(key, GraphEntry{graph, exec}).first;
  }
  cudaError_t e = cudaGraphLaunch(it->second.exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch");
  return JF_OK;
}

jf_status jf_loss_primitive_mse(jf_handle h, const void* U, const void* Uref, long long nstates, long long ncells,
                                int ncomp, double* loss_dev, void* grad, void* stream) {
  if (!h) { set_error(nullptr, "jf_loss_primitive_mse: null handle"); return JF_ERR_ARG; }
  if (!U || !Uref || !loss_dev || nstates < 1 || ncells < 1 || (ncomp != 4 && ncomp != 5) || !aligned16(U) ||
      !aligned16(Uref) || (grad && !aligned16(grad))) {
    set_error(h, "jf_loss_primitive_mse: null or misaligned array, ncomp outside {4, 5} or a non-positive count");
    return JF_ERR_ARG;
  }
  const long long total = nstates * ncells;
  const unsigned blocks = (unsigned)reduce_blocks(total, h->sms);
  const double gm1 = h->gas.gamma - 1.0;
  cudaStream_t s = (cudaStream_t)stream;
  if (h->scheme.dtype == JF_F32)
    primitive_mse_kernel<float><<<blocks, 256, 0, s>>>(static_cast<const float*>(U), static_cast<const float*>(Uref),
                                                        nstates, ncells, ncomp, gm1, h->red_loss, loss_dev,
                                                        static_cast<float*>(grad));
  else
    primitive_mse_kernel<double><<<blocks, 256, 0, s>>>(static_cast<const double*>(U),
                                                         static_cast<const double*>(Uref), nstates, ncells, ncomp,
                                                         gm1, h->red_loss, loss_dev, static_cast<double*>(grad));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "jf_loss_primitive_mse: kernel launch");
  return JF_OK;
}

jf_status jf_loss_density_l2(jf_handle h, const void* U, const void* target, double* loss_dev, void* seed,
                             void* stream) {
  if (!h || h->kind != 0) { set_error(h, "jf_loss_density_l2: not a single-grid handle"); return JF_ERR_ARG; }
  if (!U || !target || !loss_dev) { set_error(h, "jf_loss_density_l2: null pointer"); return JF_ERR_ARG; }
  return JF_DISPATCH(h, loss_impl, h, U, target, loss_dev, seed, (cudaStream_t)stream);
}

jf_status jf_set_variant(jf_handle h, int variant) {
  if (!h) { set_error(nullptr, "jf_set_variant: null handle"); return JF_ERR_ARG; }
  free_graphs(h);
  if (h->kind == 1) return batch_set_variant(h, variant);
  return JF_DISPATCH(h, select_variant, h, variant, true);
}

jf_status jf_set_nn(jf_handle h, const void* theta, int nparams) {
  if (!h) { set_error(nullptr, "jf_set_nn: null handle"); return JF_ERR_ARG; }
  if (h->scheme.flux != JF_FLUX_RUSANOV_NN) { set_error(h, "jf_set_nn: the scheme's flux is not JF_FLUX_RUSANOV_NN"); return JF_ERR_ARG; }
  if (!theta || nparams != JF_NN_PARAMS || ((uintptr_t)theta % h->esize) != 0) {
    set_error(h, "jf_set_nn: need a device array of JF_NN_PARAMS elements of the handle's dtype");
    return JF_ERR_ARG;
  }
  if (theta != h->nn) free_graphs(h);
  h->nn = theta;
  return JF_OK;
}

int jf_variant_info(jf_handle h, int variant, char* buf, int len) {
  if (!h) return JF_ERR_ARG;
  if (h->kind == 1) return batch_variant_info(h, variant, buf, len);
  return JF_DISPATCH(h, describe_variant, h, variant, buf, len);
}

int jf_auto_zchunk(int nx, int ny, int nz, int bx, int by, int ctas_per_sm, int sms) {
  if (nx < 1 || ny < 1 || nz < 1 || bx < 1 || by < 1 || ctas_per_sm < 1 || sms < 1) return 0;
  return zchunk_rule(nx, ny, nz, bx, by, ctas_per_sm, sms);
}

jf_status jf_status_sync(jf_handle h) {
  if (!h) { set_error(nullptr, "jf_status_sync: null handle"); return JF_ERR_ARG; }
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaDeviceSynchronize");
  int flag = 0;
  e = cudaMemcpy(&flag, h->flag, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaMemcpy(flag)");
  if (flag) {
    const int zero = 0;
    cudaMemcpy(h->flag, &zero, sizeof(int), cudaMemcpyHostToDevice);
    set_error(h, "a kernel met a non-physical state (rho <= 0, p <= 0 or not finite)");
    return JF_ERR_NONPHYSICAL;
  }
  return JF_OK;
}

}  // extern "C"

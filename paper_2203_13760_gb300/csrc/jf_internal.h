// Internal state of a libjf handle and the host helpers shared by the
// translation units of the library.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/jf.h"
#include "reduce.cuh"
#include "variants.h"

namespace jf {

struct GraphKey {
  const void* U;
  int nsteps;
  const void* dt;
  const void* hist;
  int variant;
  bool operator<(const GraphKey& o) const {
    return std::tie(U, nsteps, dt, hist, variant) < std::tie(o.U, o.nsteps, o.dt, o.hist, o.variant);
  }
};
struct GraphEntry {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
};


}  // namespace jf

struct jf_ctx {
  int kind = 0;              // 0: single grid, 1: batch
  jf_grid grid{};            // single grid (batch: unused)
  jf_gas gas{};
  jf_scheme scheme{};
  int dim = 1;               // active axes
  size_t esize = 4;          // bytes per element
  size_t N = 0;              // cells
  int device = 0;
  int sms = 1;
  int variant = 0;           // index into the variant list of this configuration
  int table_index = 0;       // compiled-kernel table entry
  int zchunk = 32;           // planes per CTA (3D)
  mutable std::map<long long, int> zauto;  // chosen automatic z chunk per (tile, CTAs per SM)
  void* stage[2] = {nullptr, nullptr};  // U1, U2
  void* adj[4] = {nullptr, nullptr, nullptr, nullptr};  // adjoint buffers (lazy)
  double* dt_buf = nullptr;  // device scalar
  jf::ReduceScratch* red_cfl = nullptr;
  jf::ReduceScratch* red_loss = nullptr;
  int* flag = nullptr;       // device error flag
  const void* nn = nullptr;  // Rusanov-NN parameters (caller-owned device array; jf_set_nn)
  cudaStream_t capture_stream = nullptr;
  // host-state pipeline (jf_rk3_step_host): two device buffers, the copy
  // streams and the events that order them (created at the first call)
  void* pipe_buf[2] = {nullptr, nullptr};
  cudaStream_t pipe_in = nullptr, pipe_out = nullptr;
  cudaEvent_t pipe_ev[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  std::map<jf::GraphKey, jf::GraphEntry> graphs;
  std::string err;
  // batch
  int nsim = 0;
  std::vector<jf_grid> grids;
  std::vector<void*> sim_stage;        // 2 per simulation
  void* d_sims = nullptr;              // device array of SimDesc<T> (stage.cuh)
  std::vector<unsigned char> host_desc;  // host copy of the descriptors
  // descriptor uploads: pinned staging copy, and an event recorded after every
  // graph launch and upload (work that reads the descriptors, on any stream)
  void* desc_pinned = nullptr;
  cudaEvent_t desc_done = nullptr;
  // batch adjoint: descriptors of the recompute (pinned staging, device copy,
  // event guarding the staging buffer's reuse)
  void* vjp_desc_host = nullptr;
  void* vjp_desc_dev = nullptr;
  cudaEvent_t vjp_desc_done = nullptr;
  // deferred Rusanov-NN parameter gradient (jf_batch_param_grad_begin / end):
  // face records of the adjoint steps in between, summed in one launch
  void* rec_store = nullptr;
  size_t rec_cap = 0;    // elements allocated
  size_t rec_limit = 0;  // elements of the open sweep (max_steps of the begin call)
  size_t rec_used = 0;   // elements
  bool rec_defer = false;
  void* d_cfl = nullptr;               // per-simulation CflArgs
  void* d_chunks = nullptr;            // CFL chunk list
  int nchunks = 0;
  void* d_work = nullptr;              // device work list
  int nwork = 0;
  double* d_dt = nullptr;              // per-simulation dt (internal)
  jf::ReduceScratch* d_red = nullptr;  // per-simulation reduction scratch
  std::vector<const void*> bound_ptrs; // U pointers the descriptors hold
  int batch_blocks = 0;
  int batch_rows = 0;                  // rows per work item of a row-march (ymarch) batch variant
};

namespace jf {

void set_error(jf_ctx* h, const std::string& msg);
jf_status cuda_fail(jf_ctx* h, cudaError_t e, const char* what);
int active_dims(const jf_grid& g);
jf_status check_grid(jf_ctx* h, const jf_grid& g);
jf_status check_physics(jf_ctx* h, const jf_gas& gas, const jf_scheme& s);
double spacing(const jf_grid& g, int d);
// Default tiles of 2D grids: the row tiles (rows_bx cells per row, marching
// along y) when the rows of the n grids, padded to whole tiles, cover at most
// 8 % more cells than the tile_bx x tile_by tiles do, and there are at least
// 12 rows of row tiles per resident CTA (rows_ctas_per_sm on each of sms
// SMs).  On GB300 the row tiles measured 5-11 % faster per step on large
// grids (Kelvin-Helmholtz FP32 1024^2 with 18 rows per CTA, 1536^2, 2048^2;
// FP64 1024^2, 2048^2; the 64 four-quadrant problems) and slower on small
// ones, where each CTA gets a few rows and the ring's prologue dominates
// (Kelvin-Helmholtz FP32 512^2 with 4.5 rows per CTA: 12 % slower).
bool rows_preferred(const jf_grid* grids, int n, int rows_bx, int rows_ctas_per_sm, int tile_bx, int tile_by,
                    int sms);
double conductivity(const jf_gas& gas, const jf_scheme& s);
bool dissipative(const jf_gas& gas, const jf_scheme& s);
// kernel family of a scheme: SCH_DEFAULT, SCH_GENERAL (run-time Table 2
// Godunov variants), SCH_ROE (flux splitting), their _EXT forms (slip walls
// or WENO3-JS; a walled grid with the default scheme runs SCH_GENERAL_EXT),
// or SCH_NN (Rusanov-NN)
bool has_walls(const jf_grid& g);
int scheme_kind(const jf_scheme& s, bool walls);
int scheme_kind(const jf_ctx* h);
CflArgs make_cfl(const jf_grid& g, const jf_gas& gas, const jf_scheme& s);
int reduce_blocks(long long N, int sms);
bool aligned16(const void* p);
void free_graphs(jf_ctx* h);
template <typename T> Gas<T> make_gas(const jf_gas& gas, const jf_scheme& s);
template <typename T> StageArgs<T> base_args(const jf_ctx* h);
template <typename T> jf_status launch(jf_ctx* h, const StageArgs<T>& A, cudaStream_t s);
template <typename T> jf_status select_variant(jf_ctx* h, int v, bool prepare);
template <typename T> jf_status step_impl(jf_ctx* h, void* U, const double* dt_dev, double* dt_used, cudaStream_t s);

// per-simulation CFL of a batch (jf_api.cu; the single CFL kernel)
template <typename T>
cudaError_t launch_cfl_batch(const void* sims, const void* chunks, int nchunks, const CflArgs* args,
                             ReduceScratch* red, double* dts, int* flag, cudaStream_t s);

// workspace shared by every handle kind: flag, dt scalar, reduction scratch, capture stream
jf_status alloc_common(jf_ctx* h);
void release_all(jf_ctx* h);

#ifdef JF_DEBUG_BOUNDS
// host-mapped trace buffer of the debug build (jf_common.cu), allocated at
// the first call
unsigned long long* debug_trace_dev();
#endif

// adjoint of the run-time schemes (vjp_gen.cu)
bool general_vjp_supported(const jf_ctx* h, std::string* why);
long long general_face_count(const jf_ctx* h);
template <typename T>
jf_status general_vjp(jf_ctx* h, const void* Un, const double* dt, const void* lam_out, void* lam_in, void* theta_bar,
                      cudaStream_t s);
template <typename T>
jf_status batch_general_vjp(jf_ctx* h, void* const* Un, const double* dt, void* const* lam_out, void* const* lam_in,
                            void* const* add, void* theta_bar, cudaStream_t s);
// deferred parameter gradient of a batch (jf_batch_param_grad_begin / end)
template <typename T>
jf_status batch_param_grad_begin(jf_ctx* h, int max_steps);
template <typename T>
jf_status batch_param_grad_end(jf_ctx* h, void* theta_bar, cudaStream_t s);

// batch (batch.cu)
jf_status batch_set_variant(jf_ctx* h, int variant);
int batch_variant_info(jf_ctx* h, int variant, char* buf, int len);

}  // namespace jf

// Batched simulations (jf_batch_create / jf_batch_step): many independent
// grids of uneven sizes advanced together (Section 4.5, feed_forward over a
// batch of initial buffers).
//
// Per step: one per-simulation CFL launch (each CTA reduces one chunk of
// one simulation; the last chunk of a simulation forms its dt) and the
// integrator's persistent stage launches (TVD-RK3: three, TVD-RK2: two,
// Euler: one and a copy) over the flattened (simulation, tile) work list,
// each item being one tile of the same code as the single-grid kernel.  The
// nsteps steps are captured into one CUDA graph and replayed; the graph reads
// the simulations' field pointers from device descriptors, so rebinding new
// fields only rewrites the descriptors.
#include <cstdio>
#include <cstring>
#include <vector>

#include "cfl.cuh"
#include "jf_internal.h"

namespace jf {

constexpr long long kChunk = 16384;  // cells per CFL CTA

// Euler steps of a batch: U = U1 for every simulation (blockIdx.y), the
// pointers read from the device descriptors so that rebinding stays valid.
template <typename T>
__global__ void __launch_bounds__(256) batch_copy_kernel(const SimDesc<T>* __restrict__ sims) {
  const SimDesc<T> d = sims[blockIdx.y];
  const long long n = 5 * d.N;
#ifdef JF_DEBUG_BOUNDS
  if (threadIdx.x == 0 && blockIdx.x == 0)
    jf_trace(d.trace, 0x400, blockIdx.y, (unsigned long long)d.U, (unsigned long long)d.U1, d.N, 0, 0, 0);
#endif
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    d.U[i] = d.U1[i];
}

// Trajectories (jf_batch_feed_forward): dst[s] = src[s] for every
// simulation (blockIdx.y) of one row of the pointer tables.
template <typename T>
__global__ void __launch_bounds__(256) batch_copy_pairs_kernel(const T* const* __restrict__ src,
                                                               T* const* __restrict__ dst,
                                                               const long long* __restrict__ count) {
  const T* a = src[blockIdx.y];
  T* b = dst[blockIdx.y];
  const long long n = count[blockIdx.y];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = a[i];
}

namespace {

// Batch variants: (table index, planes per work item) -- the 1D and 2D tile
// kernels once (0), the z-march kernels (3D tiles, 2D row tiles) with 32,
// 16 and 64 planes (rows) per item (the explicit z chunks of the
// single-grid variants; on the 64 four-quadrant problems 32 rows measured
// fastest: 6.34 G cell-updates/s against 6.18 with 16).
template <typename T>
std::vector<std::pair<int, int>> batch_variant_list(int dim, bool visc, int kind) {
  int count = 0;
  const StageVariant<T>* tab = stage_variants<T>(&count);
  std::vector<std::pair<int, int>> out;
  for (int i = 0; i < count; ++i)
    if (tab[i].dim == dim && tab[i].visc == visc && tab[i].scheme == kind && tab[i].launch_batch) {
      if (tab[i].ymarch || tab[i].dim == 3)
        for (int r : {32, 16, 64}) out.emplace_back(i, r);
      else
        out.emplace_back(i, 0);
    }
  return out;
}

// (Re)build the work list for the tile shape of the selected variant.
template <typename T>
jf_status setup_variant(jf_ctx* h, int v) {
  const bool visc = dissipative(h->gas, h->scheme);
  auto list = batch_variant_list<T>(h->dim, visc, scheme_kind(h));
  if (list.empty()) { set_error(h, "batch: no compiled kernel variant for this configuration"); return JF_ERR_UNSUPPORTED; }
  if (v < 0) {  // the first variant, or the first row-tile one where rows_preferred says so
    v = 0;
    int count = 0;
    const StageVariant<T>* tab = stage_variants<T>(&count);
    for (int i = 0; i < (int)list.size(); ++i)
      if (tab[list[i].first].ymarch) {
        const StageVariant<T>& r = tab[list[i].first];
        const StageVariant<T>& t0 = tab[list[0].first];
        if (rows_preferred(h->grids.data(), h->nsim, r.bx, r.minb, t0.bx, t0.by, h->sms)) v = i;
        break;
      }
  }
  if (v >= (int)list.size()) { set_error(h, "batch: variant index out of range"); return JF_ERR_ARG; }
  int count = 0;
  const StageVariant<T>* tab = stage_variants<T>(&count);
  const StageVariant<T>& sv = tab[list[v].first];
  int per_sm = 0;
  cudaError_t e = sv.prepare_batch(&per_sm);
  if (e != cudaSuccess) return cuda_fail(h, e, "batch: kernel set-up");
  if (per_sm < 1) { set_error(h, "batch: kernel does not fit on an SM"); return JF_ERR_UNSUPPORTED; }
  const long long cap = (long long)h->sms * per_sm;
  const bool march = sv.ymarch || sv.dim == 3;
  const int rows = march ? list[v].second : 1;
  std::vector<WorkItem> work;
  for (int s = 0; s < h->nsim; ++s) {
    const jf_grid& g = h->grids[s];
    // tile columns (x, y) and chunks of `rows` planes along the march (3D:
    // z; row tiles: the grid's y)
    const int tx = (g.nx + sv.bx - 1) / sv.bx;
    const int ty = sv.ymarch ? 1 : (h->dim >= 2 ? (g.ny + sv.by - 1) / sv.by : 1);
    const int marched = sv.ymarch ? g.ny : g.nz;
    const int tz = march ? (marched + rows - 1) / rows : 1;
    for (int z = 0; z < tz; ++z)
      for (int y = 0; y < ty; ++y)
        for (int x = 0; x < tx; ++x) work.push_back(WorkItem{s, x, y, z});
  }
  if (h->d_work) cudaFree(h->d_work);
  h->d_work = nullptr;
  e = cudaMalloc(&h->d_work, work.size() * sizeof(WorkItem));
  if (e != cudaSuccess) return cuda_fail(h, e, "batch: work list");
  e = cudaMemcpy(h->d_work, work.data(), work.size() * sizeof(WorkItem), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(h, e, "batch: work list");
  h->nwork = (int)work.size();
  h->batch_blocks = (int)(h->nwork < cap ? h->nwork : cap);
  h->batch_rows = rows;
  h->variant = v;
  h->table_index = list[v].first;
  return JF_OK;
}

template <typename T>
jf_status create_impl(jf_ctx* h) {
  const int ns = h->nsim;
  std::vector<SimDesc<T>> desc(ns);
  std::vector<CflArgs> cfl(ns);
  std::vector<CflChunk> chunks;
  h->sim_stage.assign(2 * ns, nullptr);
  cudaError_t e;
  // per-simulation dt first: every descriptor points at its slot
  if ((e = cudaMalloc(&h->d_dt, ns * sizeof(double))) != cudaSuccess) return cuda_fail(h, e, "batch: dt");
  if ((e = cudaMemset(h->d_dt, 0, ns * sizeof(double))) != cudaSuccess) return cuda_fail(h, e, "batch: dt");
  for (int s = 0; s < ns; ++s) {
    const jf_grid& g = h->grids[s];
    const long long N = (long long)g.nx * g.ny * g.nz;
    for (int b = 0; b < 2; ++b) {
      e = cudaMalloc(&h->sim_stage[2 * s + b], 5 * (size_t)N * sizeof(T));
      if (e != cudaSuccess) return cuda_fail(h, e, "batch: stage buffers");
    }
    SimDesc<T>& d = desc[s];
    std::memset(&d, 0, sizeof d);
    d.U = nullptr;
    d.U1 = static_cast<T*>(h->sim_stage[2 * s]);
    d.U2 = static_cast<T*>(h->sim_stage[2 * s + 1]);
    d.dt = h->d_dt + s;
    d.nx = g.nx;
    d.ny = g.ny;
    d.nz = g.nz;
    d.N = N;
#ifdef JF_DEBUG_BOUNDS
    d.trace = debug_trace_dev();
#endif
    for (int a = 0; a < 3; ++a) {
      d.periodic[a] = g.bc[2 * a] == JF_BC_PERIODIC;
      d.wall[a] = (g.bc[2 * a] == JF_BC_WALL ? 1 : 0) | (g.bc[2 * a + 1] == JF_BC_WALL ? 2 : 0);
      d.inv_h[a] = (T)(1.0 / spacing(g, a));
    }
    cfl[s] = make_cfl(g, h->gas, h->scheme);
    const int nch = (int)((N + kChunk - 1) / kChunk);
    for (int c = 0; c < nch; ++c) {
      const long long lo = c * kChunk, hi = lo + kChunk < N ? lo + kChunk : N;
      chunks.push_back(CflChunk{s, nch, lo, hi});
    }
  }
  void* p = nullptr;
  if ((e = cudaMalloc(&p, ns * sizeof(SimDesc<T>))) != cudaSuccess) return cuda_fail(h, e, "batch: descriptors");
  h->d_sims = p;
  if ((e = cudaMemcpy(p, desc.data(), ns * sizeof(SimDesc<T>), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(h, e, "batch: descriptors");
  h->host_desc.assign(reinterpret_cast<unsigned char*>(desc.data()),
                      reinterpret_cast<unsigned char*>(desc.data()) + ns * sizeof(SimDesc<T>));
  if ((e = cudaMalloc(&p, ns * sizeof(ReduceScratch))) != cudaSuccess) return cuda_fail(h, e, "batch: reduction");
  h->d_red = static_cast<ReduceScratch*>(p);
  if ((e = cudaMemset(p, 0, ns * sizeof(ReduceScratch))) != cudaSuccess) return cuda_fail(h, e, "batch: reduction");
  if ((e = cudaMalloc(&h->d_cfl, ns * sizeof(CflArgs))) != cudaSuccess) return cuda_fail(h, e, "batch: cfl");
  if ((e = cudaMemcpy(h->d_cfl, cfl.data(), ns * sizeof(CflArgs), cudaMemcpyHostToDevice)) != cudaSuccess)
    return cuda_fail(h, e, "batch: cfl");
  if ((e = cudaMalloc(&h->d_chunks, chunks.size() * sizeof(CflChunk))) != cudaSuccess)
    return cuda_fail(h, e, "batch: chunks");
  if ((e = cudaMemcpy(h->d_chunks, chunks.data(), chunks.size() * sizeof(CflChunk), cudaMemcpyHostToDevice)) !=
      cudaSuccess)
    return cuda_fail(h, e, "batch: chunks");
  h->nchunks = (int)chunks.size();
  h->bound_ptrs.assign(ns, nullptr);
  return setup_variant<T>(h, -1);
}

// Point the descriptors at the caller's fields (only when they changed).
// Every graph launch and upload records desc_done on its stream; waiting for
// it before the upload makes sure that no work queued earlier, on any stream,
// still reads the old descriptors and that the staging copy is free.  The
// upload itself is queued on s from pinned memory, so the launches that
// follow on s see the new descriptors.
template <typename T>
jf_status bind_fields(jf_ctx* h, void* const* U_ptrs, cudaStream_t s) {
  bool same = true;
  for (int i = 0; i < h->nsim; ++i) same &= h->bound_ptrs[i] == U_ptrs[i];
  if (same) return JF_OK;
  SimDesc<T>* desc = reinterpret_cast<SimDesc<T>*>(h->host_desc.data());
  for (int i = 0; i < h->nsim; ++i) desc[i].U = static_cast<T*>(U_ptrs[i]);
  const size_t bytes = h->nsim * sizeof(SimDesc<T>);
  cudaError_t e = cudaSuccess;
  if (!h->desc_pinned) e = cudaMallocHost(&h->desc_pinned, bytes);
  if (e == cudaSuccess && !h->desc_done) e = cudaEventCreateWithFlags(&h->desc_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventSynchronize(h->desc_done);
  if (e == cudaSuccess) {
    std::memcpy(h->desc_pinned, desc, bytes);
    e = cudaMemcpyAsync(h->d_sims, h->desc_pinned, bytes, cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = cudaEventRecord(h->desc_done, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "batch: descriptor update");
  for (int i = 0; i < h->nsim; ++i) h->bound_ptrs[i] = U_ptrs[i];
  return JF_OK;
}

// One batch stage (code as in batch_stage_args) over every simulation.
// FP32: the persistent kernel over the (simulation, tile) work list, reading
// the device descriptors.  FP64: one launch of the single-grid form per
// simulation (the same tile code and arithmetic), with arguments built from
// the host copy of the descriptors; the persistent FP64 form raised an
// illegal-address fault whose cause is not found, although its inputs read
// back from the device were correct.
template <typename T>
cudaError_t launch_batch_stage(jf_ctx* h, const StageVariant<T>& sv, const SimDesc<T>* dev_sims,
                               const SimDesc<T>* host_sims, int code, const Gas<T>& g, cudaStream_t s) {
  if constexpr (sizeof(T) == 8) {
    for (int i = 0; i < h->nsim; ++i) {
      StageArgs<T> A{};
      batch_stage_args(host_sims[i], code, A);
      if (sv.ymarch || sv.dim == 3) A.zchunk = h->batch_rows;
      A.flag = h->flag;
#ifdef JF_DEBUG_BOUNDS
      A.trace = debug_trace_dev();
#endif
      const cudaError_t e = sv.launch(A, g, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  } else {
    return sv.launch_batch(dev_sims, static_cast<const WorkItem*>(h->d_work), h->nwork, code, g, h->flag,
                           h->batch_blocks, h->batch_rows, s);
  }
}

template <typename T>
jf_status enqueue_steps(jf_ctx* h, int nsteps, double* dt_out, cudaStream_t s) {
  int count = 0;
  const StageVariant<T>* tab = stage_variants<T>(&count);
  const StageVariant<T>& sv = tab[h->table_index];
  Gas<T> g = make_gas<T>(h->gas, h->scheme);
  if (h->scheme.flux == JF_FLUX_RUSANOV_NN) {
    if (!h->nn) { set_error(h, "Rusanov-NN flux: no network parameters (jf_set_nn)"); return JF_ERR_ARG; }
    g.nn = static_cast<const T*>(h->nn);
  }
  const SimDesc<T>* sims = reinterpret_cast<const SimDesc<T>*>(h->d_sims);
  const SimDesc<T>* host_sims = reinterpret_cast<const SimDesc<T>*>(h->host_desc.data());
  for (int step = 0; step < nsteps; ++step) {
    cudaError_t e = launch_cfl_batch<T>(sims, h->d_chunks, h->nchunks, static_cast<const CflArgs*>(h->d_cfl),
                                        h->d_red, h->d_dt, h->flag, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "batch: cfl launch");
    // stage codes of the batch kernel: RK3 1, 2, 3; RK2 1, 4; Euler 1 + copy
    const int integ = h->scheme.integrator;
    const int codes[3] = {1, integ == JF_RK2 ? 4 : 2, 3};
    const int nst = integ == JF_RK3 ? 3 : (integ == JF_RK2 ? 2 : 1);
    for (int q = 0; q < nst; ++q) {
      e = launch_batch_stage<T>(h, sv, sims, host_sims, codes[q], g, s);
      if (e != cudaSuccess) return cuda_fail(h, e, "batch: stage launch");
    }
    if (integ == JF_EULER) {
      batch_copy_kernel<T><<<dim3((unsigned)h->sms, (unsigned)h->nsim), 256, 0, s>>>(sims);
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, e, "batch: copy launch");
    }
  }
  if (dt_out) {
    cudaError_t e = cudaMemcpyAsync(dt_out, h->d_dt, h->nsim * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "batch: dt copy");
  }
  return JF_OK;
}

// feed_forward (Section 4.5): trajectory slot 0 = U0, slot t + 1 = one step of
// slot t with the fixed per-simulation dt, for t < nsteps.  Per step: copy
// slot t to slot t + 1, then the integrator's stages in place on slot t + 1
// (descriptor row t points the simulations' U there).  Direct launches: the
// trajectory pointers are new at every call.
template <typename T>
jf_status feed_forward_batch(jf_ctx* h, void* const* U0_ptrs, void* const* traj_ptrs, int nsteps,
                             const double* dt_dev, cudaStream_t s) {
  const int ns = h->nsim;
  const size_t rows = (size_t)nsteps + 1;
  const SimDesc<T>* base = reinterpret_cast<const SimDesc<T>*>(h->host_desc.data());
  std::vector<SimDesc<T>> desc((size_t)nsteps * ns);
  std::vector<const T*> src(rows * ns);
  std::vector<T*> dst(rows * ns);
  std::vector<long long> count(ns);
  for (int i = 0; i < ns; ++i) {
    const long long n5 = 5 * base[i].N;
    count[i] = n5;
    T* traj = static_cast<T*>(traj_ptrs[i]);
    src[i] = static_cast<const T*>(U0_ptrs[i]);
    dst[i] = traj;
    for (int t = 0; t < nsteps; ++t) {
      src[(size_t)(t + 1) * ns + i] = traj + (size_t)t * n5;
      dst[(size_t)(t + 1) * ns + i] = traj + (size_t)(t + 1) * n5;
      SimDesc<T> d = base[i];
      d.U = traj + (size_t)(t + 1) * n5;
      d.dt = dt_dev + i;
      desc[(size_t)t * ns + i] = d;
    }
  }
  // one allocation for the tables; freed after the stream has used them
  const size_t bytes_desc = desc.size() * sizeof(SimDesc<T>), bytes_ptr = rows * ns * sizeof(void*);
  const size_t bytes = bytes_desc + 2 * bytes_ptr + ns * sizeof(long long);
  std::vector<unsigned char> host(bytes);
  std::memcpy(host.data(), desc.data(), bytes_desc);
  std::memcpy(host.data() + bytes_desc, src.data(), bytes_ptr);
  std::memcpy(host.data() + bytes_desc + bytes_ptr, dst.data(), bytes_ptr);
  std::memcpy(host.data() + bytes_desc + 2 * bytes_ptr, count.data(), ns * sizeof(long long));
  unsigned char* dev = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&dev), bytes, s);
  if (e != cudaSuccess) return cuda_fail(h, e, "feed_forward: tables");
  e = cudaMemcpyAsync(dev, host.data(), bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host staging buffer is local
  if (e != cudaSuccess) { cudaFreeAsync(dev, s); return cuda_fail(h, e, "feed_forward: tables"); }
  const SimDesc<T>* d_desc = reinterpret_cast<const SimDesc<T>*>(dev);
  const T* const* d_src = reinterpret_cast<const T* const*>(dev + bytes_desc);
  T* const* d_dst = reinterpret_cast<T* const*>(dev + bytes_desc + bytes_ptr);
  const long long* d_count = reinterpret_cast<const long long*>(dev + bytes_desc + 2 * bytes_ptr);
  int count_v = 0;
  const StageVariant<T>* tab = stage_variants<T>(&count_v);
  const StageVariant<T>& sv = tab[h->table_index];
  Gas<T> g = make_gas<T>(h->gas, h->scheme);
  if (h->scheme.flux == JF_FLUX_RUSANOV_NN) g.nn = static_cast<const T*>(h->nn);
  const int integ = h->scheme.integrator;
  const int codes[3] = {1, integ == JF_RK2 ? 4 : 2, 3};
  const int nst = integ == JF_RK3 ? 3 : (integ == JF_RK2 ? 2 : 1);
  const dim3 cgrid((unsigned)h->sms, (unsigned)ns);
  jf_status st = JF_OK;
  // row 0 of the copy tables: U0 -> slot 0; row t + 1: slot t -> slot t + 1
  batch_copy_pairs_kernel<T><<<cgrid, 256, 0, s>>>(d_src, d_dst, d_count);
  if ((e = cudaGetLastError()) != cudaSuccess) st = cuda_fail(h, e, "feed_forward: copy launch");
  for (int t = 0; t < nsteps && st == JF_OK; ++t) {
    batch_copy_pairs_kernel<T><<<cgrid, 256, 0, s>>>(d_src + (size_t)(t + 1) * ns, d_dst + (size_t)(t + 1) * ns,
                                                     d_count);
    if ((e = cudaGetLastError()) != cudaSuccess) { st = cuda_fail(h, e, "feed_forward: copy launch"); break; }
    const SimDesc<T>* sims = d_desc + (size_t)t * ns;  // U = slot t + 1
    for (int q = 0; q < nst; ++q) {
      e = launch_batch_stage<T>(h, sv, sims, desc.data() + (size_t)t * ns, codes[q], g, s);
      if (e != cudaSuccess) { st = cuda_fail(h, e, "feed_forward: stage launch"); break; }
    }
    if (st == JF_OK && integ == JF_EULER) {
      batch_copy_kernel<T><<<cgrid, 256, 0, s>>>(sims);
      if ((e = cudaGetLastError()) != cudaSuccess) st = cuda_fail(h, e, "feed_forward: copy launch");
    }
  }
  cudaFreeAsync(dev, s);
  return st;
}

template <typename T>
jf_status step_batch(jf_ctx* h, void* const* U_ptrs, int nsteps, double* dt_out, cudaStream_t s) {
  bool rebound = false;
  for (int i = 0; i < h->nsim; ++i) rebound |= h->bound_ptrs[i] != U_ptrs[i];
  jf_status st = bind_fields<T>(h, U_ptrs, s);
  if (st != JF_OK) return st;
  // the FP64 stage launches carry the field pointers in their arguments
  if (sizeof(T) == 8 && rebound) free_graphs(h);
  const GraphKey key{nullptr, nsteps, dt_out, nullptr, h->variant};
  auto it = h->graphs.find(key);
  if (it == h->graphs.end()) {
    cudaStream_t cs = h->capture_stream;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamBeginCapture");
    st = enqueue_steps<T>(h, nsteps, dt_out, cs);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(cs, &graph);
    if (st != JF_OK) { if (graph) cudaGraphDestroy(graph); return st; }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return cuda_fail(h, e, "cudaGraphInstantiate"); }
    it = h->graphs.emplace(key, GraphEntry{graph, exec}).first;
  }
  cudaError_t e = cudaGraphLaunch(it->second.exec, s);
  if (e == cudaSuccess) e = cudaEventRecord(h->desc_done, s);  // the graph reads the descriptors
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch");
  return JF_OK;
}

}  // namespace

jf_status batch_set_variant(jf_ctx* h, int variant) {
  return h->scheme.dtype == JF_F32 ? setup_variant<float>(h, variant) : setup_variant<double>(h, variant);
}

int batch_variant_info(jf_ctx* h, int variant, char* buf, int len) {
  const bool visc = dissipative(h->gas, h->scheme);
  std::vector<std::pair<int, int>> list;
  int bx = 0, by = 0, rows = 0;
  bool ymarch = false, dim3d = false;
  auto get = [&](const auto* tab) {
    if (variant >= 0 && variant < (int)list.size()) {
      const auto& sv = tab[list[variant].first];
      bx = sv.bx;
      by = sv.by;
      ymarch = sv.ymarch;
      dim3d = sv.dim == 3;
      rows = list[variant].second;
    }
  };
  int c = 0;
  if (h->scheme.dtype == JF_F32) {
    list = batch_variant_list<float>(h->dim, visc, scheme_kind(h));
    get(stage_variants<float>(&c));
  } else {
    list = batch_variant_list<double>(h->dim, visc, scheme_kind(h));
    get(stage_variants<double>(&c));
  }
  if (variant >= 0 && variant < (int)list.size() && buf && len > 0) {
    if (ymarch)
      std::snprintf(buf, (size_t)len, "tile=%dx%d ymarch rows=%d persistent", bx, by, rows);
    else if (dim3d)
      std::snprintf(buf, (size_t)len, "tile=%dx%d zchunk=%d persistent", bx, by, rows);
    else
      std::snprintf(buf, (size_t)len, "tile=%dx%d persistent", bx, by);
  }
  return (int)list.size();
}

}  // namespace jf

using namespace jf;

extern "C" {

jf_status jf_batch_create(const jf_grid* grids, int nsim, const jf_gas* gas, const jf_scheme* scheme,
                          jf_handle* out) {
  if (!grids || !gas || !scheme || !out || nsim < 1 || nsim > 65535) {
    set_error(nullptr, "jf_batch_create: null argument or nsim outside 1..65535");
    return JF_ERR_ARG;
  }
  *out = nullptr;
  jf_status st;
  if ((st = check_physics(nullptr, *gas, *scheme)) != JF_OK) return st;
  const int dim = active_dims(grids[0]);
  for (int s = 0; s < nsim; ++s) {
    if ((st = check_grid(nullptr, grids[s])) != JF_OK) return st;
    if (active_dims(grids[s]) != dim) {
      set_error(nullptr, "jf_batch_create: all simulations must have the same number of active axes");
      return JF_ERR_UNSUPPORTED;
    }
  }
  jf_ctx* h = new jf_ctx();
  h->kind = 1;
  h->gas = *gas;
  h->scheme = *scheme;
  h->grid = grids[0];
  h->dim = dim;
  h->esize = scheme->dtype == JF_F32 ? 4 : 8;
  h->nsim = nsim;
  h->grids.assign(grids, grids + nsim);
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e != cudaSuccess) { st = cuda_fail(nullptr, e, "jf_batch_create: device query"); delete h; return st; }
  st = alloc_common(h);
  if (st == JF_OK) st = scheme->dtype == JF_F32 ? create_impl<float>(h) : create_impl<double>(h);
  if (st != JF_OK) {
    if (!h->err.empty()) set_error(nullptr, h->err);
    jf_destroy(h);
    return st;
  }
  *out = h;
  return JF_OK;
}

jf_status jf_batch_feed_forward(jf_handle h, void* const* U0_ptrs, void* const* traj_ptrs, int nsteps,
                                const double* dt_dev, void* stream) {
  if (!h || h->kind != 1) { set_error(h, "jf_batch_feed_forward: not a batch handle"); return JF_ERR_ARG; }
  if (!U0_ptrs || !traj_ptrs || !dt_dev || nsteps < 0) {
    set_error(h, "jf_batch_feed_forward: null argument or nsteps < 0");
    return JF_ERR_ARG;
  }
  if (h->scheme.flux == JF_FLUX_RUSANOV_NN && !h->nn) {
    set_error(h, "Rusanov-NN flux: no network parameters (jf_set_nn)");
    return JF_ERR_ARG;
  }
  for (int s = 0; s < h->nsim; ++s)
    if (!U0_ptrs[s] || !traj_ptrs[s] || !aligned16(U0_ptrs[s]) || !aligned16(traj_ptrs[s])) {
      set_error(h, "jf_batch_feed_forward: every state and trajectory must be a 16-byte aligned device array");
      return JF_ERR_ARG;
    }
  return h->scheme.dtype == JF_F32
             ? feed_forward_batch<float>(h, U0_ptrs, traj_ptrs, nsteps, dt_dev, (cudaStream_t)stream)
             : feed_forward_batch<double>(h, U0_ptrs, traj_ptrs, nsteps, dt_dev, (cudaStream_t)stream);
}

jf_status jf_batch_step(jf_handle h, void* const* U_ptrs, int nsteps, double* dt_dev, void* stream) {
  if (!h || h->kind != 1) { set_error(h, "jf_batch_step: not a batch handle"); return JF_ERR_ARG; }
  if (!U_ptrs || nsteps < 0) { set_error(h, "jf_batch_step: bad arguments"); return JF_ERR_ARG; }
  for (int s = 0; s < h->nsim; ++s)
    if (!U_ptrs[s] || !aligned16(U_ptrs[s])) {
      set_error(h, "jf_batch_step: every field must be a 16-byte aligned device array");
      return JF_ERR_ARG;
    }
  if (nsteps == 0) return JF_OK;
  return h->scheme.dtype == JF_F32 ? step_batch<float>(h, U_ptrs, nsteps, dt_dev, (cudaStream_t)stream)
                                   : step_batch<double>(h, U_ptrs, nsteps, dt_dev, (cudaStream_t)stream);
}

}  // extern "C"

#ifdef JF_DEBUG_BOUNDS
// Device-side inputs of a batch's kernels read back without launching any
// kernel (debug build only; not declared in jf.h): info = {nwork,
// batch_blocks, table_index, bx, by, threads, smem, scheme}; the work list;
// the descriptors after binding U_ptrs.
extern "C" int jf_debug_batch_inputs(jf_handle h, void* const* U_ptrs, int* info, void* work, int work_len,
                                     void* sims, int sims_len) {
  if (!h || h->kind != 1) return -1;
  info[0] = h->nwork;
  info[1] = h->batch_blocks;
  info[2] = h->table_index;
  int count = 0;
  if (h->scheme.dtype == JF_F32) {
    const StageVariant<float>& v = stage_variants<float>(&count)[h->table_index];
    info[3] = v.bx; info[4] = v.by; info[5] = v.threads; info[6] = (int)v.smem; info[7] = v.scheme;
    if (bind_fields<float>(h, U_ptrs, nullptr) != JF_OK) return -2;
  } else {
    const StageVariant<double>& v = stage_variants<double>(&count)[h->table_index];
    info[3] = v.bx; info[4] = v.by; info[5] = v.threads; info[6] = (int)v.smem; info[7] = v.scheme;
    if (bind_fields<double>(h, U_ptrs, nullptr) != JF_OK) return -2;
  }
  const int wb = h->nwork * (int)sizeof(WorkItem), sb = (int)h->host_desc.size();
  if (work_len < wb || sims_len < sb) return -3;
  if (cudaMemcpy(work, h->d_work, (size_t)wb, cudaMemcpyDeviceToHost) != cudaSuccess) return -4;
  if (cudaMemcpy(sims, h->d_sims, (size_t)sb, cudaMemcpyDeviceToHost) != cudaSuccess) return -4;
  return 0;
}

// Host copy of a batch's descriptors (debug build only; not declared in jf.h).
extern "C" int jf_debug_batch_desc(jf_handle h, void* buf, int len) {
  if (!h || h->kind != 1) return -1;
  const int n = (int)h->host_desc.size();
  if (buf && len >= n) std::memcpy(buf, h->host_desc.data(), (size_t)n);
  return n;
}
#endif

// Adjoint of one fixed-dt step for the run-time schemes (vjp_gen.cuh): slip
// walls, WENO5-JS / WENO3-JS, HLLC (Einfeldt speeds) or the Rusanov-NN flux,
// TVD-RK3, TVD-RK2 or Euler, inviscid; for one grid (jf_rk3_step_vjp,
// jf_rk3_step_vjp_params) or every simulation of a batch in the same launches
// (jf_batch_step_vjp).  With V(U, m) = m + dt J(U)^T m and l = lam_out:
//   TVD-RK3 (as vjp.cu): l2 = V(U2, 2/3 l); l1 = V(U1, 1/4 l2); ln = 1/3 l + 3/4 l2 + V(Un, l1);
//   TVD-RK2 (U1 = Un + dt L(Un); U^{n+1} = 1/2 Un + 1/2 (U1 + dt L(U1))):
//            l1 = V(U1, 1/2 l); ln = 1/2 l + V(Un, l1);
//   Euler:   ln = V(Un, l);
// plus an optional addend of ln (the loss cotangent at U^n in a trajectory
// sweep).  With the Rusanov-NN flux every V also adds its parameter gradient
// sum_f abar_f d alpha_f / d theta to theta_bar (when given).
#include <cstring>
#include <vector>

#include "jf_internal.h"
#include "vjp_gen.cuh"

namespace jf {

namespace {

// Geometry of one grid for the per-face adjoint (pointers and factors unset).
template <typename T>
GVjpArgs<T> grid_args(const jf_grid& grid, int dim) {
  GVjpArgs<T> A;
  std::memset(&A, 0, sizeof A);
  const int n[3] = {grid.nx, grid.ny, grid.nz};
  for (int a = 0; a < 3; ++a) {
    A.n[a] = n[a];
    A.periodic[a] = grid.bc[2 * a] == JF_BC_PERIODIC;
    A.wall[a] = (grid.bc[2 * a] == JF_BC_WALL ? 1 : 0) | (grid.bc[2 * a + 1] == JF_BC_WALL ? 2 : 0);
    A.inv_h[a] = (T)(1.0 / spacing(grid, a));
  }
  A.N = (long long)n[0] * n[1] * n[2];
  for (int a = 0; a < dim; ++a) {
    long long c = 1;
    for (int e = 0; e < 3; ++e) c *= e == a ? (long long)n[e] + (A.periodic[a] ? 0 : 1) : n[e];
    A.nface[a] = c;
  }
  return A;
}

template <typename T>
long long faces_of(const GVjpArgs<T>& A) { return A.nface[0] + A.nface[1] + A.nface[2]; }

template <typename T, int DIM, int RECON, int FLUX>
cudaError_t launch_face(const GVjpBatch<T>& B, const Gas<T>& g, long long nf, cudaStream_t s) {
  constexpr size_t smem = gvjp_face_smem_bytes<T, FLUX>();
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(gvjp_face_kernel<T, DIM, RECON, FLUX>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const long long blocks = (nf + kGvjpThreads - 1) / kGvjpThreads;
  gvjp_face_kernel<T, DIM, RECON, FLUX><<<(unsigned)blocks, kGvjpThreads, smem, s>>>(B, g);
  return cudaGetLastError();
}

template <typename T, int DIM>
cudaError_t launch_face_dim(const GVjpBatch<T>& B, const Gas<T>& g, long long nf, int recon, bool nn,
                            cudaStream_t s) {
  if (recon == JF_WENO3_JS)
    return nn ? launch_face<T, DIM, 2, 4>(B, g, nf, s) : launch_face<T, DIM, 2, 0>(B, g, nf, s);
  return nn ? launch_face<T, DIM, 0, 4>(B, g, nf, s) : launch_face<T, DIM, 0, 0>(B, g, nf, s);
}

// One V over the grids `sims` (their pointers and factors set): the point,
// face and (Rusanov-NN with theta_bar) parameter-gradient launches, in chunks
// of GVjpBatch::kMax grids.  The grids' records are consecutive from the
// first grid's rec.
template <typename T>
jf_status gvjp_stage(jf_ctx* h, const Gas<T>& g, std::vector<GVjpArgs<T>>& sims, T* theta_bar, cudaStream_t s) {
  const bool nn = h->scheme.flux == JF_FLUX_RUSANOV_NN;
  const int recon = h->scheme.recon;
  for (size_t c0 = 0; c0 < sims.size(); c0 += GVjpBatch<T>::kMax) {
    GVjpBatch<T> B;
    std::memset(&B, 0, sizeof B);
    B.nsim = (int)std::min<size_t>(GVjpBatch<T>::kMax, sims.size() - c0);
    for (int k = 0; k < B.nsim; ++k) {
      B.sim[k] = sims[c0 + k];
      if (!nn) B.sim[k].rec = nullptr;
      B.face_base[k + 1] = B.face_base[k] + faces_of(B.sim[k]);
      B.cell_base[k + 1] = B.cell_base[k] + B.sim[k].N;
    }
    const long long nf = B.face_base[B.nsim];
    gvjp_point_kernel<T><<<reduce_blocks(B.cell_base[B.nsim], h->sms), 256, 0, s>>>(B);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "adjoint: point launch");
    e = h->dim == 1 ? launch_face_dim<T, 1>(B, g, nf, recon, nn, s)
                    : (h->dim == 2 ? launch_face_dim<T, 2>(B, g, nf, recon, nn, s)
                                   : launch_face_dim<T, 3>(B, g, nf, recon, nn, s));
    if (e != cudaSuccess) return cuda_fail(h, e, "adjoint: face launch");
    if (nn && theta_bar) {
      const long long chunks = (nf + 31) / 32;
      const long long blocks = std::min<long long>((chunks + kNnWarps - 1) / kNnWarps, 2LL * h->sms);
      nn_param_grad_kernel<T><<<(unsigned)blocks, 32 * kNnWarps, nn_grad_smem_bytes<T>(), s>>>(
          g.nn, B.sim[0].rec, nf, theta_bar);
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, e, "adjoint: parameter-gradient launch");
    }
  }
  return JF_OK;
}

// Per-grid state of one adjoint step: the step's inputs and its buffers.
template <typename T>
struct StepPtrs {
  const T* Un;
  const T* lam;    // lam_out
  T* lam_in;
  const T* add;    // added to lam_in (may be null)
  const double* dt;
  T* U1;
  T* U2;
  T* l1;
  T* l2;
  T* rec;
};

// Stages of one step of the integrator.
int step_stages(const jf_ctx* h) {
  return h->scheme.integrator == JF_RK3 ? 3 : (h->scheme.integrator == JF_RK2 ? 2 : 1);
}

// The integrator's chain over the grids (geometry in `geo`, one entry per grid).
// The face records of stage j (in the chain's order) start rec_stride * j
// elements after P[k].rec (0: every stage reuses the same records).
template <typename T>
jf_status gvjp_chain(jf_ctx* h, const Gas<T>& g, const std::vector<GVjpArgs<T>>& geo,
                     const std::vector<StepPtrs<T>>& P, T* theta_bar, size_t rec_stride, cudaStream_t s) {
  const int integ = h->scheme.integrator;
  std::vector<GVjpArgs<T>> V(geo);
  size_t stage = 0;  // stages set up so far, counted per grid 0
  auto set = [&](size_t k, const T* Us, const T* lam, T s_in, const T* x1, T a1, const T* x2, T a2, const T* x3,
                 T a3, T* out) {
    GVjpArgs<T>& A = V[k];
    A.Us = Us; A.lam = lam; A.s_in = s_in; A.x1 = x1; A.a1 = a1; A.x2 = x2; A.a2 = a2; A.x3 = x3; A.a3 = a3;
    A.out = out; A.dt = P[k].dt;
    if (k == 0) ++stage;
    A.rec = P[k].rec ? P[k].rec + rec_stride * (stage - 1) : nullptr;
  };
  jf_status st;
  if (integ == JF_RK3) {
    for (size_t k = 0; k < V.size(); ++k)
      set(k, P[k].U2, P[k].lam, T(2.0 / 3.0), nullptr, T(0), nullptr, T(0), nullptr, T(0), P[k].l2);
    if ((st = gvjp_stage<T>(h, g, V, theta_bar, s)) != JF_OK) return st;
    for (size_t k = 0; k < V.size(); ++k)
      set(k, P[k].U1, P[k].l2, T(0.25), nullptr, T(0), nullptr, T(0), nullptr, T(0), P[k].l1);
    if ((st = gvjp_stage<T>(h, g, V, theta_bar, s)) != JF_OK) return st;
    for (size_t k = 0; k < V.size(); ++k)
      set(k, P[k].Un, P[k].l1, T(1), P[k].lam, T(1.0 / 3.0), P[k].l2, T(0.75), P[k].add, T(1), P[k].lam_in);
    return gvjp_stage<T>(h, g, V, theta_bar, s);
  }
  if (integ == JF_RK2) {
    for (size_t k = 0; k < V.size(); ++k)
      set(k, P[k].U1, P[k].lam, T(0.5), nullptr, T(0), nullptr, T(0), nullptr, T(0), P[k].l1);
    if ((st = gvjp_stage<T>(h, g, V, theta_bar, s)) != JF_OK) return st;
    for (size_t k = 0; k < V.size(); ++k)
      set(k, P[k].Un, P[k].l1, T(1), P[k].lam, T(0.5), P[k].add, T(1), nullptr, T(0), P[k].lam_in);
    return gvjp_stage<T>(h, g, V, theta_bar, s);
  }
  for (size_t k = 0; k < V.size(); ++k)
    set(k, P[k].Un, P[k].lam, T(1), P[k].add, T(1), nullptr, T(0), nullptr, T(0), P[k].lam_in);
  return gvjp_stage<T>(h, g, V, theta_bar, s);
}

// Forward recompute of one grid's stage states with the stage kernels of the
// step (single-grid form of the handle's table entry).
template <typename T>
jf_status recompute(jf_ctx* h, const StageVariant<T>& sv, const Gas<T>& g, StageArgs<T> A, const StepPtrs<T>& p,
                    cudaStream_t s) {
  const int integ = h->scheme.integrator;
  if (integ == JF_EULER) return JF_OK;
  A.dt = p.dt;
  A.Us = p.Un; A.Un = nullptr; A.out = p.U1; A.a = T(0); A.b = T(1);
  cudaError_t e = sv.launch(A, g, s);
  if (e == cudaSuccess && integ == JF_RK3) {
    A.Us = p.U1; A.Un = p.Un; A.out = p.U2; A.a = T(0.75); A.b = T(0.25);
    e = sv.launch(A, g, s);
  }
  return e == cudaSuccess ? JF_OK : cuda_fail(h, e, "adjoint: forward recompute");
}

template <typename T>
jf_status network(jf_ctx* h, Gas<T>& g) {
  if (h->scheme.flux != JF_FLUX_RUSANOV_NN) return JF_OK;
  if (!h->nn) { set_error(h, "Rusanov-NN flux: no network parameters (jf_set_nn)"); return JF_ERR_ARG; }
  g.nn = static_cast<const T*>(h->nn);
  return JF_OK;
}

template <typename T>
jf_status prepare_param_grad(jf_ctx* h, const void* theta_bar) {
  static_assert(nn_grad_smem_bytes<T>() <= 227 * 1024, "parameter-gradient tile exceeds shared memory");
  if (!theta_bar) return JF_OK;
  const cudaError_t e = cudaFuncSetAttribute(nn_param_grad_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)nn_grad_smem_bytes<T>());
  return e == cudaSuccess ? JF_OK : cuda_fail(h, e, "adjoint: kernel set-up");
}

}  // namespace

long long general_face_count(const jf_ctx* h) { return faces_of(grid_args<double>(h->grid, h->dim)); }

bool general_vjp_supported(const jf_ctx* h, std::string* why) {
  const jf_scheme& s = h->scheme;
  if (dissipative(h->gas, s)) { *why = "viscous and heat fluxes have an adjoint only in the default scheme without walls"; return false; }
  if (s.recon != JF_WENO5_JS && s.recon != JF_WENO3_JS) { *why = "the adjoint reconstructions are WENO5-JS and WENO3-JS"; return false; }
  if (s.flux == JF_FLUX_RUSANOV_NN) return true;
  if (s.flux == JF_FLUX_HLLC && s.signal_speed == JF_EINFELDT) return true;
  *why = "the adjoint fluxes are HLLC with Einfeldt speeds and Rusanov-NN";
  return false;
}

template <typename T>
jf_status general_vjp(jf_ctx* h, const void* Un, const double* dt, const void* lam_out, void* lam_in, void* theta_bar,
                      cudaStream_t s) {
  const GVjpArgs<T> geo = grid_args<T>(h->grid, h->dim);
  for (int i = 0; i < 3; ++i) {
    const size_t bytes = i < 2 ? 5 * h->N * sizeof(T) : (size_t)faces_of(geo) * 5 * sizeof(T);
    if (!h->adj[i]) {
      cudaError_t e = cudaMalloc(&h->adj[i], bytes);
      if (e != cudaSuccess) return cuda_fail(h, e, "adjoint: buffers");
    }
  }
  jf_status st;
  if ((st = prepare_param_grad<T>(h, theta_bar)) != JF_OK) return st;
  Gas<T> g = make_gas<T>(h->gas, h->scheme);
  if ((st = network<T>(h, g)) != JF_OK) return st;
  StepPtrs<T> p{static_cast<const T*>(Un), static_cast<const T*>(lam_out), static_cast<T*>(lam_in), nullptr, dt,
                static_cast<T*>(h->stage[0]), static_cast<T*>(h->stage[1]), static_cast<T*>(h->adj[1]),
                static_cast<T*>(h->adj[0]), static_cast<T*>(h->adj[2])};
  int count = 0;
  const StageVariant<T>& sv = stage_variants<T>(&count)[h->table_index];
  if ((st = recompute<T>(h, sv, g, base_args<T>(h), p, s)) != JF_OK) return st;
  return gvjp_chain<T>(h, g, std::vector<GVjpArgs<T>>{geo}, std::vector<StepPtrs<T>>{p},
                       static_cast<T*>(theta_bar), 0, s);
}

// Forward recompute of every grid's stage states in one launch per stage
// (FP32: the persistent batch kernel over the handle's work list, with a
// descriptor row whose U is each grid's Un and whose dt is its step, staged
// through pinned memory; FP64: the single-grid form per grid, as the batch's
// forward runs).
template <typename T>
jf_status recompute_batch(jf_ctx* h, const StageVariant<T>& sv, const Gas<T>& g, const std::vector<StepPtrs<T>>& P,
                          cudaStream_t s) {
  const SimDesc<T>* desc = reinterpret_cast<const SimDesc<T>*>(h->host_desc.data());
  const int ns = h->nsim, integ = h->scheme.integrator;
  if (integ == JF_EULER) return JF_OK;
  if constexpr (sizeof(T) == 8) {
    for (int k = 0; k < ns; ++k) {
      StageArgs<T> A{};
      batch_stage_args(desc[k], 1, A);
      A.flag = h->flag;
      jf_status st = recompute<T>(h, sv, g, A, P[k], s);
      if (st != JF_OK) return st;
    }
    return JF_OK;
  } else {
    const size_t bytes = (size_t)ns * sizeof(SimDesc<T>);
    cudaError_t e = cudaSuccess;
    if (!h->vjp_desc_host) {
      if ((e = cudaMallocHost(&h->vjp_desc_host, bytes)) != cudaSuccess) return cuda_fail(h, e, "batch adjoint: staging");
      if ((e = cudaMalloc(&h->vjp_desc_dev, bytes)) != cudaSuccess) return cuda_fail(h, e, "batch adjoint: descriptors");
      if ((e = cudaEventCreateWithFlags(&h->vjp_desc_done, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(h, e, "batch adjoint: event");
    } else if ((e = cudaEventSynchronize(h->vjp_desc_done)) != cudaSuccess) {
      return cuda_fail(h, e, "batch adjoint: staging reuse");
    }
    SimDesc<T>* row = static_cast<SimDesc<T>*>(h->vjp_desc_host);
    for (int k = 0; k < ns; ++k) {
      row[k] = desc[k];
      row[k].U = const_cast<T*>(P[k].Un);
      row[k].dt = P[k].dt;
    }
    e = cudaMemcpyAsync(h->vjp_desc_dev, row, bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(h->vjp_desc_done, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "batch adjoint: descriptor upload");
    const SimDesc<T>* dev = static_cast<const SimDesc<T>*>(h->vjp_desc_dev);
    e = sv.launch_batch(dev, static_cast<const WorkItem*>(h->d_work), h->nwork, 1, g, h->flag, h->batch_blocks,
                        h->batch_rows, s);
    if (e == cudaSuccess && integ == JF_RK3)
      e = sv.launch_batch(dev, static_cast<const WorkItem*>(h->d_work), h->nwork, 2, g, h->flag, h->batch_blocks,
                          h->batch_rows, s);
    return e == cudaSuccess ? JF_OK : cuda_fail(h, e, "batch adjoint: forward recompute");
  }
}

template <typename T>
jf_status batch_general_vjp(jf_ctx* h, void* const* Un, const double* dt, void* const* lam_out, void* const* lam_in,
                            void* const* add, void* theta_bar, cudaStream_t s) {
  const int ns = h->nsim;
  std::vector<GVjpArgs<T>> geo(ns);
  size_t pool = 0;
  for (int k = 0; k < ns; ++k) {
    geo[k] = grid_args<T>(h->grids[k], h->dim);
    pool += (size_t)(10 * geo[k].N + 5 * faces_of(geo[k]));
  }
  if (!h->adj[0]) {  // l1, l2 of every grid, then every grid's face records
    cudaError_t e = cudaMalloc(&h->adj[0], pool * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(h, e, "batch adjoint: buffers");
  }
  jf_status st;
  if ((st = prepare_param_grad<T>(h, theta_bar)) != JF_OK) return st;
  Gas<T> g = make_gas<T>(h->gas, h->scheme);
  if ((st = network<T>(h, g)) != JF_OK) return st;
  int count = 0;
  const StageVariant<T>& sv = stage_variants<T>(&count)[h->table_index];
  const SimDesc<T>* desc = reinterpret_cast<const SimDesc<T>*>(h->host_desc.data());
  std::vector<StepPtrs<T>> P(ns);
  T* lbuf = static_cast<T*>(h->adj[0]);
  size_t off = 0;
  for (int k = 0; k < ns; ++k) off += 10 * (size_t)geo[k].N;
  T* rbuf = lbuf + off;  // records of all grids, consecutive
  size_t faces = 0;
  for (int k = 0; k < ns; ++k) faces += (size_t)faces_of(geo[k]);
  const bool defer = h->rec_defer && theta_bar && h->scheme.flux == JF_FLUX_RUSANOV_NN;
  const size_t rec_step = (size_t)step_stages(h) * 5 * faces;  // record elements of one step
  if (defer) {
    if (h->rec_used + rec_step > h->rec_limit) {
      set_error(h, "jf_batch_step_vjp: the record store of jf_batch_param_grad_begin is full (more steps than "
                   "max_steps)");
      return JF_ERR_ARG;
    }
    rbuf = static_cast<T*>(h->rec_store) + h->rec_used;
  }
  off = 0;
  size_t roff = 0;
  for (int k = 0; k < ns; ++k) {
    P[k] = StepPtrs<T>{static_cast<const T*>(Un[k]), static_cast<const T*>(lam_out[k]), static_cast<T*>(lam_in[k]),
                       add ? static_cast<const T*>(add[k]) : nullptr, dt + k, desc[k].U1, desc[k].U2,
                       lbuf + off, lbuf + off + 5 * geo[k].N, rbuf + roff};
    off += 10 * (size_t)geo[k].N;
    roff += 5 * (size_t)faces_of(geo[k]);
  }
  if ((st = recompute_batch<T>(h, sv, g, P, s)) != JF_OK) return st;
  if (!defer) return gvjp_chain<T>(h, g, geo, P, static_cast<T*>(theta_bar), 0, s);
  // deferred parameter gradient: the records stay in the store for
  // jf_batch_param_grad_end, one region per stage
  if ((st = gvjp_chain<T>(h, g, geo, P, nullptr, rec_step / step_stages(h), s)) != JF_OK) return st;
  h->rec_used += rec_step;
  return JF_OK;
}

template <typename T>
jf_status batch_param_grad_begin(jf_ctx* h, int max_steps) {
  size_t faces = 0;
  for (int k = 0; k < h->nsim; ++k) faces += (size_t)faces_of(grid_args<T>(h->grids[k], h->dim));
  const size_t need = (size_t)max_steps * step_stages(h) * 5 * faces;
  if (need > h->rec_cap) {
    if (h->rec_store) cudaFree(h->rec_store);
    h->rec_store = nullptr;
    h->rec_cap = 0;
    const cudaError_t e = cudaMalloc(&h->rec_store, need * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(h, e, "jf_batch_param_grad_begin: record store");
    h->rec_cap = need;
  }
  h->rec_limit = need;
  h->rec_used = 0;
  h->rec_defer = true;
  return JF_OK;
}

template <typename T>
jf_status batch_param_grad_end(jf_ctx* h, void* theta_bar, cudaStream_t s) {
  const long long n = (long long)(h->rec_used / 5);
  h->rec_defer = false;
  h->rec_used = 0;
  if (n == 0) return JF_OK;
  jf_status st;
  if ((st = prepare_param_grad<T>(h, theta_bar)) != JF_OK) return st;
  Gas<T> g = make_gas<T>(h->gas, h->scheme);
  if ((st = network<T>(h, g)) != JF_OK) return st;
  const long long chunks = (n + 31) / 32;
  const long long blocks = std::min<long long>((chunks + kNnWarps - 1) / kNnWarps, 2LL * h->sms);
  nn_param_grad_kernel<T><<<(unsigned)blocks, 32 * kNnWarps, nn_grad_smem_bytes<T>(), s>>>(
      g.nn, static_cast<const T*>(h->rec_store), n, static_cast<T*>(theta_bar));
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? JF_OK : cuda_fail(h, e, "jf_batch_param_grad_end: launch");
}

template jf_status general_vjp<float>(jf_ctx*, const void*, const double*, const void*, void*, void*, cudaStream_t);
template jf_status general_vjp<double>(jf_ctx*, const void*, const double*, const void*, void*, void*, cudaStream_t);
template jf_status batch_general_vjp<float>(jf_ctx*, void* const*, const double*, void* const*, void* const*,
                                            void* const*, void*, cudaStream_t);
template jf_status batch_general_vjp<double>(jf_ctx*, void* const*, const double*, void* const*, void* const*,
                                             void* const*, void*, cudaStream_t);
template jf_status batch_param_grad_begin<float>(jf_ctx*, int);
template jf_status batch_param_grad_begin<double>(jf_ctx*, int);
template jf_status batch_param_grad_end<float>(jf_ctx*, void*, cudaStream_t);
template jf_status batch_param_grad_end<double>(jf_ctx*, void*, cudaStream_t);

}  // namespace jf

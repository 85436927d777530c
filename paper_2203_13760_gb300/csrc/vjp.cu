// Adjoint of one fixed-dt TVD-RK3 step (jf_rk3_step_vjp), Section 7.2:
// gradients propagated back through the solver.
//
// Forward:  U1 = Un + dt L(Un); U2 = 3/4 Un + 1/4 (U1 + dt L(U1));
//           U3 = 1/3 Un + 2/3 (U2 + dt L(U2)).
// Backward, with l3 = dLoss/dU3 and V(U, m) = m + dt J(U)^T m:
//   l2 = V(U2, 2/3 l3);  l1 = V(U1, 1/4 l2);
//   ln = 1/3 l3 + 3/4 l2 + V(Un, l1).
// U1 and U2 are recomputed with the forward stage kernel (dt fixed, not
// differentiated), or taken from the caller (jf_rk3_step_vjp_stages, after
// jf_rk3_step_keep kept them); l2 and l1 live in two adjoint buffers
// allocated at the first call of a handle.
#include "jf_internal.h"
#include "vjp_inst.cuh"

namespace jf {

// the configurations of the fused stage-VJP kernel: the default scheme
// (HLLC, Einfeldt speeds, WENO5-JS, TVD-RK3) without walls
static bool fused_vjp(const jf_ctx* h) {
  const jf_scheme& sc = h->scheme;
  return sc.flux == JF_FLUX_HLLC && sc.recon == JF_WENO5_JS && sc.signal_speed == JF_EINFELDT &&
         sc.integrator == JF_RK3 && !has_walls(h->grid);
}

// The three stage-VJP launches of one step, from the stage states U0, U1, U2.
template <typename T>
jf_status vjp_backward(jf_ctx* h, const T* U0, const T* U1, const T* U2, const double* dt, const void* lam_out,
                       void* lam_in, cudaStream_t s) {
  VjpLaunch<T> L = vjp_launcher<T>(h->dim, dissipative(h->gas, h->scheme));
  if (!L) { set_error(h, "jf_rk3_step_vjp: no adjoint kernel for this configuration"); return JF_ERR_UNSUPPORTED; }
  for (int i = 0; i < 2; ++i)
    if (!h->adj[i]) {
      cudaError_t e = cudaMalloc(&h->adj[i], 5 * h->N * sizeof(T));
      if (e != cudaSuccess) return cuda_fail(h, e, "jf_rk3_step_vjp: adjoint buffers");
    }
  if (h->dim == 3 && !h->adj[3]) {  // the z-marching kernel's accumulator of W (+T) cotangents
    cudaError_t e = cudaMalloc(&h->adj[3], 6 * h->N * sizeof(T));
    if (e != cudaSuccess) return cuda_fail(h, e, "jf_rk3_step_vjp: adjoint accumulator");
  }
  T* l2 = static_cast<T*>(h->adj[0]);
  T* l1 = static_cast<T*>(h->adj[1]);
  T* scratch = static_cast<T*>(h->adj[3]);
  VjpArgs<T> V;
  V.n[0] = h->grid.nx;
  V.n[1] = h->grid.ny;
  V.n[2] = h->grid.nz;
  V.N = (long long)h->N;
  for (int a = 0; a < 3; ++a) {
    V.periodic[a] = h->grid.bc[2 * a] == JF_BC_PERIODIC;
    V.inv_h[a] = (T)(1.0 / spacing(h->grid, a));
  }
  V.dt = dt;
  V.flag = h->flag;
  const Gas<T> g = make_gas<T>(h->gas, h->scheme);
  struct Call { const T* Us; const T* lam; T s_in; const T* x1; T a1; const T* x2; T a2; T* out; };
  const Call calls[3] = {
      {U2, static_cast<const T*>(lam_out), T(2.0 / 3.0), nullptr, T(0), nullptr, T(0), l2},
      {U1, l2, T(0.25), nullptr, T(0), nullptr, T(0), l1},
      {U0, l1, T(1), static_cast<const T*>(lam_out), T(1.0 / 3.0), l2, T(0.75), static_cast<T*>(lam_in)},
  };
  for (const Call& c : calls) {
    V.Us = c.Us; V.lam = c.lam; V.s_in = c.s_in; V.x1 = c.x1; V.a1 = c.a1; V.x2 = c.x2; V.a2 = c.a2; V.out = c.out;
    cudaError_t e = L(V, g, scratch, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "jf_rk3_step_vjp: kernel launch");
  }
  return JF_OK;
}

// One fixed-dt TVD-RK3 step of U in place with the stage states written to
// U1o and U2o (the launches of step_impl with other output buffers).
template <typename T>
jf_status step_keep(jf_ctx* h, void* U, const double* dt, void* U1o, void* U2o, cudaStream_t s) {
  T* Un = static_cast<T*>(U);
  T* U1 = static_cast<T*>(U1o);
  T* U2 = static_cast<T*>(U2o);
  StageArgs<T> A = base_args<T>(h);
  A.dt = dt;
  jf_status st;
  A.Us = Un; A.Un = nullptr; A.out = U1; A.a = T(0); A.b = T(1);
  if ((st = launch<T>(h, A, s)) != JF_OK) return st;
  A.Us = U1; A.Un = Un; A.out = U2; A.a = T(0.75); A.b = T(0.25);
  if ((st = launch<T>(h, A, s)) != JF_OK) return st;
  A.Us = U2; A.Un = Un; A.out = Un; A.a = T(1.0 / 3.0); A.b = T(2.0 / 3.0);
  return launch<T>(h, A, s);
}

template <typename T>
jf_status vjp_impl(jf_ctx* h, const void* Un, const double* dt, const void* lam_out, void* lam_in,
                   cudaStream_t s) {
  if (!fused_vjp(h)) {
    // the run-time schemes: the per-face adjoint of vjp_gen.cu
    std::string why;
    if (!general_vjp_supported(h, &why)) {
      set_error(h, "jf_rk3_step_vjp: " + why);
      return JF_ERR_UNSUPPORTED;
    }
    return general_vjp<T>(h, Un, dt, lam_out, lam_in, nullptr, s);
  }
  if (!vjp_launcher<T>(h->dim, dissipative(h->gas, h->scheme))) {
    set_error(h, "jf_rk3_step_vjp: no adjoint kernel for this configuration");
    return JF_ERR_UNSUPPORTED;
  }
  const T* U0 = static_cast<const T*>(Un);
  T* U1 = static_cast<T*>(h->stage[0]);
  T* U2 = static_cast<T*>(h->stage[1]);
  // forward recompute of the stage states
  StageArgs<T> A = base_args<T>(h);
  A.dt = dt;
  A.Us = U0; A.Un = nullptr; A.out = U1; A.a = T(0); A.b = T(1);
  jf_status st = launch<T>(h, A, s);
  if (st != JF_OK) return st;
  A.Us = U1; A.Un = U0; A.out = U2; A.a = T(0.75); A.b = T(0.25);
  if ((st = launch<T>(h, A, s)) != JF_OK) return st;
  return vjp_backward<T>(h, U0, U1, U2, dt, lam_out, lam_in, s);
}

}  // namespace jf

using namespace jf;

extern "C" jf_status jf_rk3_step_vjp(jf_handle h, const void* Un, const double* dt_dev, const void* lam_out,
                                     void* lam_in, void* stream) {
  if (!h || h->kind != 0) { set_error(h, "jf_rk3_step_vjp: not a single-grid handle"); return JF_ERR_ARG; }
  if (!Un || !dt_dev || !lam_out || !lam_in || !aligned16(Un) || !aligned16(lam_out) || !aligned16(lam_in) ||
      lam_in == lam_out || lam_in == Un) {
    set_error(h, "jf_rk3_step_vjp: bad arguments (dt_dev is required; lam_in must differ from lam_out and Un)");
    return JF_ERR_ARG;
  }
  return h->scheme.dtype == JF_F32
             ? vjp_impl<float>(h, Un, dt_dev, lam_out, lam_in, (cudaStream_t)stream)
             : vjp_impl<double>(h, Un, dt_dev, lam_out, lam_in, (cudaStream_t)stream);
}

extern "C" jf_status jf_rk3_step_keep(jf_handle h, void* U_inout, const double* dt_dev, void* U1_out, void* U2_out,
                                      void* stream) {
  if (!h || h->kind != 0) { set_error(h, "jf_rk3_step_keep: not a single-grid handle"); return JF_ERR_ARG; }
  if (h->scheme.integrator != JF_RK3) {
    set_error(h, "jf_rk3_step_keep: the scheme's integrator is not TVD-RK3");
    return JF_ERR_UNSUPPORTED;
  }
  if (!U_inout || !dt_dev || !U1_out || !U2_out || !aligned16(U_inout) || !aligned16(U1_out) || !aligned16(U2_out) ||
      U1_out == U_inout || U2_out == U_inout || U1_out == U2_out) {
    set_error(h, "jf_rk3_step_keep: bad arguments (dt_dev is required; U, U1_out and U2_out must be distinct)");
    return JF_ERR_ARG;
  }
  return h->scheme.dtype == JF_F32 ? step_keep<float>(h, U_inout, dt_dev, U1_out, U2_out, (cudaStream_t)stream)
                                   : step_keep<double>(h, U_inout, dt_dev, U1_out, U2_out, (cudaStream_t)stream);
}

extern "C" jf_status jf_rk3_step_vjp_stages(jf_handle h, const void* Un, const void* U1, const void* U2,
                                            const double* dt_dev, const void* lam_out, void* lam_in, void* stream) {
  if (!h || h->kind != 0) { set_error(h, "jf_rk3_step_vjp_stages: not a single-grid handle"); return JF_ERR_ARG; }
  if (!fused_vjp(h)) {
    set_error(h, "jf_rk3_step_vjp_stages: only the default scheme (HLLC, Einfeldt, WENO5-JS, TVD-RK3) without walls");
    return JF_ERR_UNSUPPORTED;
  }
  if (!Un || !U1 || !U2 || !dt_dev || !lam_out || !lam_in || !aligned16(Un) || !aligned16(U1) || !aligned16(U2) ||
      !aligned16(lam_out) || !aligned16(lam_in) || lam_in == lam_out || lam_in == Un || lam_in == U1 ||
      lam_in == U2) {
    set_error(h, "jf_rk3_step_vjp_stages: bad arguments (dt_dev is required; lam_in must differ from the other arrays)");
    return JF_ERR_ARG;
  }
  return h->scheme.dtype == JF_F32
             ? vjp_backward<float>(h, static_cast<const float*>(Un), static_cast<const float*>(U1),
                                   static_cast<const float*>(U2), dt_dev, lam_out, lam_in, (cudaStream_t)stream)
             : vjp_backward<double>(h, static_cast<const double*>(Un), static_cast<const double*>(U1),
                                    static_cast<const double*>(U2), dt_dev, lam_out, lam_in, (cudaStream_t)stream);
}

extern "C" jf_status jf_rk3_step_vjp_params(jf_handle h, const void* Un, const double* dt_dev, const void* lam_out,
                                            void* lam_in, void* theta_bar, void* stream) {
  if (!h || h->kind != 0) { set_error(h, "jf_rk3_step_vjp_params: not a single-grid handle"); return JF_ERR_ARG; }
  if (h->scheme.flux != JF_FLUX_RUSANOV_NN) {
    set_error(h, "jf_rk3_step_vjp_params: the scheme's flux is not JF_FLUX_RUSANOV_NN");
    return JF_ERR_ARG;
  }
  if (!Un || !dt_dev || !lam_out || !lam_in || !theta_bar || !aligned16(Un) || !aligned16(lam_out) ||
      !aligned16(lam_in) || lam_in == lam_out || lam_in == Un || ((uintptr_t)theta_bar % h->esize) != 0) {
    set_error(h, "jf_rk3_step_vjp_params: bad arguments (dt_dev and theta_bar are required; lam_in must differ "
                 "from lam_out and Un)");
    return JF_ERR_ARG;
  }
  std::string why;
  if (!general_vjp_supported(h, &why)) { set_error(h, "jf_rk3_step_vjp_params: " + why); return JF_ERR_UNSUPPORTED; }
  return h->scheme.dtype == JF_F32
             ? general_vjp<float>(h, Un, dt_dev, lam_out, lam_in, theta_bar, (cudaStream_t)stream)
             : general_vjp<double>(h, Un, dt_dev, lam_out, lam_in, theta_bar, (cudaStream_t)stream);
}

extern "C" jf_status jf_batch_step_vjp(jf_handle h, void* const* Un_ptrs, const double* dt_dev,
                                       void* const* lam_out_ptrs, void* const* lam_in_ptrs, void* const* add_ptrs,
                                       void* theta_bar, void* stream) {
  if (!h || h->kind != 1) { set_error(h, "jf_batch_step_vjp: not a batch handle"); return JF_ERR_ARG; }
  if (!Un_ptrs || !dt_dev || !lam_out_ptrs || !lam_in_ptrs) {
    set_error(h, "jf_batch_step_vjp: null argument");
    return JF_ERR_ARG;
  }
  for (int s = 0; s < h->nsim; ++s) {
    const void* a = add_ptrs ? add_ptrs[s] : nullptr;
    if (!Un_ptrs[s] || !lam_out_ptrs[s] || !lam_in_ptrs[s] || !aligned16(Un_ptrs[s]) || !aligned16(lam_out_ptrs[s]) ||
        !aligned16(lam_in_ptrs[s]) || (a && !aligned16(a)) || lam_in_ptrs[s] == lam_out_ptrs[s] ||
        lam_in_ptrs[s] == Un_ptrs[s]) {
      set_error(h, "jf_batch_step_vjp: every Un / lam_out / lam_in must be a 16-byte aligned device array, and "
                   "lam_in must differ from lam_out and Un");
      return JF_ERR_ARG;
    }
  }
  if (theta_bar && (h->scheme.flux != JF_FLUX_RUSANOV_NN || ((uintptr_t)theta_bar % h->esize) != 0)) {
    set_error(h, "jf_batch_step_vjp: theta_bar needs the JF_FLUX_RUSANOV_NN flux (and element alignment)");
    return JF_ERR_ARG;
  }
  std::string why;
  if (!general_vjp_supported(h, &why)) { set_error(h, "jf_batch_step_vjp: " + why); return JF_ERR_UNSUPPORTED; }
  return h->scheme.dtype == JF_F32
             ? batch_general_vjp<float>(h, Un_ptrs, dt_dev, lam_out_ptrs, lam_in_ptrs, add_ptrs, theta_bar,
                                        (cudaStream_t)stream)
             : batch_general_vjp<double>(h, Un_ptrs, dt_dev, lam_out_ptrs, lam_in_ptrs, add_ptrs, theta_bar,
                                         (cudaStream_t)stream);
}

extern "C" jf_status jf_batch_param_grad_begin(jf_handle h, int max_steps) {
  if (!h || h->kind != 1) { set_error(h, "jf_batch_param_grad_begin: not a batch handle"); return JF_ERR_ARG; }
  if (h->scheme.flux != JF_FLUX_RUSANOV_NN || max_steps < 1) {
    set_error(h, "jf_batch_param_grad_begin: needs the JF_FLUX_RUSANOV_NN flux and max_steps >= 1");
    return JF_ERR_ARG;
  }
  return h->scheme.dtype == JF_F32 ? batch_param_grad_begin<float>(h, max_steps)
                                   : batch_param_grad_begin<double>(h, max_steps);
}

extern "C" jf_status jf_batch_param_grad_end(jf_handle h, void* theta_bar, void* stream) {
  if (!h || h->kind != 1) { set_error(h, "jf_batch_param_grad_end: not a batch handle"); return JF_ERR_ARG; }
  if (!h->rec_defer || !theta_bar || ((uintptr_t)theta_bar % h->esize) != 0) {
    set_error(h, "jf_batch_param_grad_end: needs a preceding jf_batch_param_grad_begin and an aligned theta_bar");
    return JF_ERR_ARG;
  }
  return h->scheme.dtype == JF_F32 ? batch_param_grad_end<float>(h, theta_bar, (cudaStream_t)stream)
                                   : batch_param_grad_end<double>(h, theta_bar, (cudaStream_t)stream);
}

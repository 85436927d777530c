// Adjoint of one fixed-dt TVD-RK3 step (jf_rk3_step_vjp), Section 7.2:
// gradients propagated back through the solver.
//
// Forward:  U1 = Un + dt L(Un); U2 = 3/4 Un + 1/4 (U1 + dt L(U1));
//           U3 = 1/3 Un + 2/3 (U2 + dt L(U2)).
// Backward, with l3 = dLoss/dU3 and V(U, m) = m + dt J(U)^T m:
//   l2 = V(U2, 2/3 l3);  l1 = V(U1, 1/4 l2);
//   ln = 1/3 l3 + 3/4 l2 + V(Un, l1).
// U1 and U2 are recomputed with the forward stage kernel (dt fixed, not
// differentiated); l2 and l1 live in two adjoint buffers allocated at the
// first call of a handle.
#include "jf_internal.h"
#include "vjp_inst.cuh"

namespace jf {

template <typename T>
jf_status vjp_impl(jf_ctx* h, const void* Un, const double* dt, const void* lam_out, void* lam_in,
                   cudaStream_t s) {
  const bool visc = dissipative(h->gas, h->scheme);
  const jf_scheme& sc = h->scheme;
  if (sc.flux != JF_FLUX_HLLC || sc.recon != JF_WENO5_JS || sc.signal_speed != JF_EINFELDT ||
      sc.integrator != JF_RK3 || has_walls(h->grid)) {
    // the run-time schemes: the per-face adjoint of vjp_gen.cu
    std::string why;
    if (!general_vjp_supported(h, &why)) {
      set_error(h, "jf_rk3_step_vjp: " + why);
      return JF_ERR_UNSUPPORTED;
    }
    return general_vjp<T>(h, Un, dt, lam_out, lam_in, nullptr, s);
  }
  VjpLaunch<T> L = vjp_launcher<T>(h->dim, visc);
  if (!L) { set_error(h, "jf_rk3_step_vjp: no adjoint kernel for this configuration"); return JF_ERR_UNSUPPORTED; }
  for (int i = 0; i < 2; ++i)
    if (!h->adj[i]) {
      cudaError_t e = cudaMalloc(&h->adj[i], 5 * h->N * sizeof(T));
      if (e != cudaSuccess) return cuda_fail(h, e, "jf_rk3_step_vjp: adjoint buffers");
    }
  const T* U0 = static_cast<const T*>(Un);
  T* U1 = static_cast<T*>(h->stage[0]);
  T* U2 = static_cast<T*>(h->stage[1]);
  T* l2 = static_cast<T*>(h->adj[0]);
  T* l1 = static_cast<T*>(h->adj[1]);
  // forward recompute of the stage states
  StageArgs<T> A = base_args<T>(h);
  A.dt = dt;
  A.Us = U0; A.Un = nullptr; A.out = U1; A.a = T(0); A.b = T(1);
  jf_status st = launch<T>(h, A, s);
  if (st != JF_OK) return st;
  A.Us = U1; A.Un = U0; A.out = U2; A.a = T(0.75); A.b = T(0.25);
  if ((st = launch<T>(h, A, s)) != JF_OK) return st;
  // backward
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
    cudaError_t e = L(V, g, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "jf_rk3_step_vjp: kernel launch");
  }
  return JF_OK;
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

// Adjoint of one fixed-dt step for the run-time schemes (vjp_gen.cuh): slip
// walls, WENO5-JS / WENO3-JS, HLLC (Einfeldt speeds) or the Rusanov-NN flux,
// TVD-RK3, TVD-RK2 or Euler, inviscid.  With V(U, m) = m + dt J(U)^T m:
//   TVD-RK3 (as vjp.cu): l2 = V(U2, 2/3 l); l1 = V(U1, 1/4 l2); ln = 1/3 l + 3/4 l2 + V(Un, l1);
//   TVD-RK2 (U1 = Un + dt L(Un); U^{n+1} = 1/2 Un + 1/2 (U1 + dt L(U1))):
//            l1 = V(U1, 1/2 l); ln = 1/2 l + V(Un, l1);
//   Euler:   ln = V(Un, l).
// With the Rusanov-NN flux every V also adds its parameter gradient
// sum_f abar_f d alpha_f / d theta to theta_bar (when given).
#include <cstring>

#include "jf_internal.h"
#include "vjp_gen.cuh"

namespace jf {

namespace {

template <typename T, int DIM, int RECON, int FLUX>
cudaError_t launch_face(const GVjpArgs<T>& A, const Gas<T>& g, long long nf, cudaStream_t s) {
  constexpr size_t smem = gvjp_face_smem_bytes<T, FLUX>();
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(gvjp_face_kernel<T, DIM, RECON, FLUX>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const long long blocks = (nf + kGvjpThreads - 1) / kGvjpThreads;
  gvjp_face_kernel<T, DIM, RECON, FLUX><<<(unsigned)blocks, kGvjpThreads, smem, s>>>(A, g);
  return cudaGetLastError();
}

template <typename T, int DIM>
cudaError_t launch_face_dim(const GVjpArgs<T>& A, const Gas<T>& g, long long nf, int recon, bool nn, cudaStream_t s) {
  if (recon == JF_WENO3_JS)
    return nn ? launch_face<T, DIM, 2, 4>(A, g, nf, s) : launch_face<T, DIM, 2, 0>(A, g, nf, s);
  return nn ? launch_face<T, DIM, 0, 4>(A, g, nf, s) : launch_face<T, DIM, 0, 0>(A, g, nf, s);
}

// One V launch: out = a1 x1 + a2 x2 + m + dt J(Us)^T m, m = s_in lam (and the
// parameter gradient of the network into theta_bar when given).
template <typename T>
jf_status gvjp_stage(jf_ctx* h, const Gas<T>& g, const T* Us, const T* lam, T s_in, const T* x1, T a1, const T* x2,
                     T a2, T* out, const double* dt, T* rec, T* theta_bar, cudaStream_t s) {
  GVjpArgs<T> A;
  std::memset(&A, 0, sizeof A);
  A.Us = Us; A.lam = lam; A.x1 = x1; A.x2 = x2; A.out = out; A.dt = dt;
  A.s_in = s_in; A.a1 = a1; A.a2 = a2;
  const int nn3[3] = {h->grid.nx, h->grid.ny, h->grid.nz};
  long long nf = 0;
  for (int a = 0; a < 3; ++a) {
    A.n[a] = nn3[a];
    A.periodic[a] = h->grid.bc[2 * a] == JF_BC_PERIODIC;
    A.wall[a] = (h->grid.bc[2 * a] == JF_BC_WALL ? 1 : 0) | (h->grid.bc[2 * a + 1] == JF_BC_WALL ? 2 : 0);
    A.inv_h[a] = (T)(1.0 / spacing(h->grid, a));
  }
  A.N = (long long)h->N;
  for (int a = 0; a < h->dim; ++a) {
    long long c = 1;
    for (int e = 0; e < 3; ++e) c *= e == a ? (long long)nn3[e] + (A.periodic[a] ? 0 : 1) : nn3[e];
    A.nface[a] = c;
    nf += c;
  }
  const bool nn = h->scheme.flux == JF_FLUX_RUSANOV_NN;
  A.rec = nn ? rec : nullptr;
  gvjp_point_kernel<T><<<reduce_blocks(5 * A.N, h->sms), 256, 0, s>>>(A);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "adjoint: point launch");
  const int recon = h->scheme.recon;
  e = h->dim == 1 ? launch_face_dim<T, 1>(A, g, nf, recon, nn, s)
                  : (h->dim == 2 ? launch_face_dim<T, 2>(A, g, nf, recon, nn, s)
                                 : launch_face_dim<T, 3>(A, g, nf, recon, nn, s));
  if (e != cudaSuccess) return cuda_fail(h, e, "adjoint: face launch");
  if (nn && theta_bar) {
    nn_param_grad_kernel<T><<<(unsigned)((nf + 31) / 32), 32, nn_grad_smem_bytes<T>(), s>>>(g.nn, rec, nf, theta_bar);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(h, e, "adjoint: parameter-gradient launch");
  }
  return JF_OK;
}

}  // namespace

long long general_face_count(const jf_ctx* h) {
  const int n[3] = {h->grid.nx, h->grid.ny, h->grid.nz};
  long long nf = 0;
  for (int a = 0; a < h->dim; ++a) {
    long long c = 1;
    for (int e = 0; e < 3; ++e) c *= e == a ? (long long)n[e] + (h->grid.bc[2 * a] == JF_BC_PERIODIC ? 0 : 1) : n[e];
    nf += c;
  }
  return nf;
}

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
  const long long nf = general_face_count(h);
  static_assert(nn_grad_smem_bytes<T>() <= 227 * 1024, "parameter-gradient tile exceeds shared memory");
  if (theta_bar) {
    cudaError_t e = cudaFuncSetAttribute(nn_param_grad_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)nn_grad_smem_bytes<T>());
    if (e != cudaSuccess) return cuda_fail(h, e, "adjoint: kernel set-up");
  }
  for (int i = 0; i < 3; ++i) {
    const size_t bytes = i < 2 ? 5 * h->N * sizeof(T) : (size_t)nf * 5 * sizeof(T);
    if (!h->adj[i]) {
      cudaError_t e = cudaMalloc(&h->adj[i], bytes);
      if (e != cudaSuccess) return cuda_fail(h, e, "adjoint: buffers");
    }
  }
  Gas<T> g = make_gas<T>(h->gas, h->scheme);
  if (h->scheme.flux == JF_FLUX_RUSANOV_NN) {
    if (!h->nn) { set_error(h, "Rusanov-NN flux: no network parameters (jf_set_nn)"); return JF_ERR_ARG; }
    g.nn = static_cast<const T*>(h->nn);
  }
  const T* U0 = static_cast<const T*>(Un);
  const T* L = static_cast<const T*>(lam_out);
  T* Lin = static_cast<T*>(lam_in);
  T* U1 = static_cast<T*>(h->stage[0]);
  T* U2 = static_cast<T*>(h->stage[1]);
  T* l2 = static_cast<T*>(h->adj[0]);
  T* l1 = static_cast<T*>(h->adj[1]);
  T* rec = static_cast<T*>(h->adj[2]);
  T* tb = static_cast<T*>(theta_bar);
  // forward recompute of the stage states (same kernels as the step)
  StageArgs<T> A = base_args<T>(h);
  A.dt = dt;
  jf_status st;
  const int integ = h->scheme.integrator;
  if (integ != JF_EULER) {
    A.Us = U0; A.Un = nullptr; A.out = U1; A.a = T(0); A.b = T(1);
    if ((st = launch<T>(h, A, s)) != JF_OK) return st;
  }
  if (integ == JF_RK3) {
    A.Us = U1; A.Un = U0; A.out = U2; A.a = T(0.75); A.b = T(0.25);
    if ((st = launch<T>(h, A, s)) != JF_OK) return st;
    if ((st = gvjp_stage<T>(h, g, U2, L, T(2.0 / 3.0), nullptr, T(0), nullptr, T(0), l2, dt, rec, tb, s)) != JF_OK)
      return st;
    if ((st = gvjp_stage<T>(h, g, U1, l2, T(0.25), nullptr, T(0), nullptr, T(0), l1, dt, rec, tb, s)) != JF_OK)
      return st;
    return gvjp_stage<T>(h, g, U0, l1, T(1), L, T(1.0 / 3.0), l2, T(0.75), Lin, dt, rec, tb, s);
  }
  if (integ == JF_RK2) {
    if ((st = gvjp_stage<T>(h, g, U1, L, T(0.5), nullptr, T(0), nullptr, T(0), l1, dt, rec, tb, s)) != JF_OK)
      return st;
    return gvjp_stage<T>(h, g, U0, l1, T(1), L, T(0.5), nullptr, T(0), Lin, dt, rec, tb, s);
  }
  return gvjp_stage<T>(h, g, U0, L, T(1), nullptr, T(0), nullptr, T(0), Lin, dt, rec, tb, s);
}

template jf_status general_vjp<float>(jf_ctx*, const void*, const double*, const void*, void*, void*, cudaStream_t);
template jf_status general_vjp<double>(jf_ctx*, const void*, const double*, const void*, void*, void*, cudaStream_t);

}  // namespace jf

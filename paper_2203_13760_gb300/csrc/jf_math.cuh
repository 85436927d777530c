// Point-wise numerics of the finite-volume stage, shared by the forward,
// batched and adjoint kernels of libjf.
//
// References (arXiv 2203.13760):
//   primitives        Section 2, Eq. (StiffenedGas) with B = 0
//   weno5             Section 3.3 (High-order Godunov approach, step 1),
//                     WENO5-JS of Jiang & Shu (1996) or WENO5-Z of Borges et
//                     al. (2008) (Table 2)
//   hllc              Section 3.3 steps 2-3, Eq. (ApproxRiemannSolver): HLLC
//                     (Toro 1994) with Einfeldt (1988), Davis (1988) or Toro
//                     (1994) signal speeds (Table 2)
//   hll, rusanov      Table 2: HLL (Harten, Lax, van Leer 1983) and local
//                     Lax-Friedrichs
//   rusanov_nn        Section 7.4: Rusanov flux with a learned dissipation
//   weno3             Table 2 WENO3-JS
//   df4 / dc4 / rc4   Section 3.4 fourth-order face derivative, cell-centre
//                     derivative and central interpolation to the face
#pragma once
#include <cuda_runtime.h>

// point-wise numerics compile for the host too (used by host-side checks)
#define JF_HD __host__ __device__ __forceinline__

namespace jf {

template <typename T>
struct Gas {
  T gamma;     // ratio of specific heats
  T gm1;       // gamma - 1
  T inv_gm1;   // 1 / (gamma - 1)
  T inv_R;     // 1 / R
  T mu;        // dynamic viscosity (0 if inviscid)
  T lambda;    // heat conductivity
  T eps;       // WENO5 epsilon
  int safe;    // first-order fallback for non-positive reconstructed rho / p
  int flux;    // 0 HLLC, 1 HLL, 2 Rusanov (local Lax-Friedrichs), 4 Rusanov-NN
  int recon;   // 0 WENO5-JS, 1 WENO5-Z, 2 WENO3-JS
  int speeds;  // 0 Einfeldt, 1 Davis, 2 Toro (PVRS)
  const T* nn; // Rusanov-NN parameters (NN_PARAMS values; shared memory in the kernels)
};

// The Rusanov-NN dissipation network (Section 7.4): inputs
// x = (|du_n|, mean u_n, mean c, |ds|), three hidden layers of NN_HIDDEN ReLU
// units, alpha = exp(output); parameters W1 [32][4], b1, W2 [32][32], b2,
// W3 [32][32], b3, W4 [32], b4 (row-major, outputs by inputs).
constexpr int NN_HIDDEN = 32;
constexpr int NN_PARAMS = 32 * 4 + 32 + 2 * (32 * 32 + 32) + 32 + 1;

template <typename T> JF_HD T tsqrt(T x);
template <> JF_HD float tsqrt<float>(float x) { return sqrtf(x); }
template <> JF_HD double tsqrt<double>(double x) { return sqrt(x); }

// Reciprocal of the point-wise numerics.  FP32 device code takes the
// hardware approximate reciprocal (__fdividef: one MUFU operation, within
// 2 ulp for |x| < 2^126); FP64 and host code divide exactly.
template <typename T> JF_HD T trcp(T x) { return T(1) / x; }
template <> JF_HD float trcp<float>(float x) {
#ifdef __CUDA_ARCH__
  return __fdividef(1.0f, x);
#else
  return 1.0f / x;
#endif
}

template <typename T> JF_HD T tmin(T a, T b) { return b < a ? b : a; }
template <typename T> JF_HD T tmax(T a, T b) { return a < b ? b : a; }

// WENO5-JS: value at x_{i+1/2} biased to the left, from v[i-2..i+2].
// Candidate stencils q_k, smoothness indicators beta_k, weights
// alpha_k = d_k / (eps + beta_k)^2 with d = (1/10, 6/10, 3/10),
// omega_k = alpha_k / sum(alpha).
// With z != 0 the WENO5-Z weights of Borges et al. (2008) replace the JS
// ones: tau5 = |beta_0 - beta_2|, alpha_k = d_k (1 + tau5 / (eps + beta_k)).
template <typename T>
JF_HD T weno5(T vm2, T vm1, T v0, T vp1, T vp2, T eps, int z = 0) {
  const T sixth = T(1) / T(6);
  const T q0 = (T(2) * vm2 - T(7) * vm1 + T(11) * v0) * sixth;
  const T q1 = (-vm1 + T(5) * v0 + T(2) * vp1) * sixth;
  const T q2 = (T(2) * v0 + T(5) * vp1 - vp2) * sixth;
  const T c13 = T(13) / T(12);
  const T d0 = vm2 - T(2) * vm1 + v0, e0 = vm2 - T(4) * vm1 + T(3) * v0;
  const T d1 = vm1 - T(2) * v0 + vp1, e1 = vm1 - vp1;
  const T d2 = v0 - T(2) * vp1 + vp2, e2 = T(3) * v0 - T(4) * vp1 + vp2;
  const T b0 = c13 * d0 * d0 + T(0.25) * e0 * e0;
  const T b1 = c13 * d1 * d1 + T(0.25) * e1 * e1;
  const T b2 = c13 * d2 * d2 + T(0.25) * e2 * e2;
  const T t0 = eps + b0, t1 = eps + b1, t2 = eps + b2;
  if constexpr (sizeof(T) == 8) {
    // alpha_k scaled by a common product of the (eps + beta_j) terms: one
    // division instead of four (the factors are >= eps, far inside the FP64
    // range).  JS: alpha_k ~ d_k / t_k^2, scaled by (t0 t1 t2)^2; Z:
    // alpha_k ~ d_k (t_k + tau5) / t_k, scaled by t0 t1 t2.
    T a0, a1, a2;
    if (z) {
      const T tau = fabs(b0 - b2);
      a0 = T(0.1) * (t0 + tau) * t1 * t2;
      a1 = T(0.6) * (t1 + tau) * t0 * t2;
      a2 = T(0.3) * (t2 + tau) * t0 * t1;
    } else {
      const T s0 = t0 * t0, s1 = t1 * t1, s2 = t2 * t2;
      a0 = T(0.1) * s1 * s2;
      a1 = T(0.6) * s0 * s2;
      a2 = T(0.3) * s0 * s1;
    }
    return (a0 * q0 + a1 * q1 + a2 * q2) / (a0 + a1 + a2);
  } else {
    T r0, r1, r2;
    if (z) {
      const T tau = fabs(b0 - b2);
      r0 = (t0 + tau) * trcp(t0);
      r1 = (t1 + tau) * trcp(t1);
      r2 = (t2 + tau) * trcp(t2);
    } else {
      r0 = trcp(t0 * t0);
      r1 = trcp(t1 * t1);
      r2 = trcp(t2 * t2);
    }
    const T a0 = T(0.1) * r0, a1 = T(0.6) * r1, a2 = T(0.3) * r2;
    return (a0 * q0 + a1 * q1 + a2 * q2) * trcp(a0 + a1 + a2);
  }
}

// The left and right WENO5-JS states of one face component in packed FP32x2
// arithmetic (sm_100+ FFMA2 / FADD2 / FMUL2): lane x reconstructs
// (v[i-2], .., v[i+2]) -> v^-, lane y the mirrored stencil
// (v[i+3], .., v[i-1]) -> v^+.  The formula of weno5, rearranged to fewer
// operations (equal up to rounding):
//  * with the differences D1 = vm2 - vm1, D2 = v0 - vm1, D3 = vp1 - v0,
//    D4 = vp1 - vp2 the candidates are q_k = v0 + delta_k / 6 with
//    delta = (5 D2 + 2 D1, D2 + 2 D3, 4 D3 + D4), and the smoothness terms
//    are d0 = D2 + D1, d1 = D3 - D2, |d2| = |D3 + D4|, e0 = 3 D2 + D1,
//    |e1| = |D2 + D3|, |e2| = |3 D3 + D4| (only their squares enter);
//  * every eps + beta_k is scaled by 12/13 (a common factor of the three
//    alpha_k, which cancels in omega_k), so t_k = d_k^2 + 3/13 e_k^2 + 12/13 eps;
//  * with r_k = 1 / t_k^2 and alpha_k scaled by 10/3 (weights 1/3, 2, 1),
//    v^ = v0 + (r0 delta0/18 + r1 delta1/3 + r2 delta2/6) / (r0/3 + 2 r1 + r2);
//  * WENO5-Z (z != 0): r_k = (t_k + tau) / t_k with tau = |t_0 - t_2| (the
//    same 12/13 scaling of tau5 = |beta_0 - beta_2|).
__device__ __forceinline__ float2 weno5_pair(float2 vm2, float2 vm1, float2 v0, float2 vp1, float2 vp2, float eps,
                                             int z = 0) {
  auto c = [](float x) { return make_float2(x, x); };
  const float2 m1 = c(-1.0f);
  const float2 D1 = __ffma2_rn(m1, vm1, vm2);
  const float2 D2 = __ffma2_rn(m1, vm1, v0);
  const float2 D3 = __ffma2_rn(m1, v0, vp1);
  const float2 D4 = __ffma2_rn(m1, vp2, vp1);
  const float2 d0 = __fadd2_rn(D2, D1), e0 = __ffma2_rn(c(3.0f), D2, D1);
  const float2 d1 = __ffma2_rn(m1, D2, D3), e1 = __fadd2_rn(D2, D3);
  const float2 d2 = __fadd2_rn(D3, D4), e2 = __ffma2_rn(c(3.0f), D3, D4);
  const float2 k3 = c(3.0f / 13.0f), ke = c(12.0f / 13.0f * eps);
  const float2 t0 = __ffma2_rn(d0, d0, __ffma2_rn(__fmul2_rn(k3, e0), e0, ke));
  const float2 t1 = __ffma2_rn(d1, d1, __ffma2_rn(__fmul2_rn(k3, e1), e1, ke));
  const float2 t2 = __ffma2_rn(d2, d2, __ffma2_rn(__fmul2_rn(k3, e2), e2, ke));
  // approximate reciprocals (t_k^2 >= (12/13 eps)^2 > 0, so the sum is > 0)
  auto rcp2 = [](float2 x) { return make_float2(__fdividef(1.0f, x.x), __fdividef(1.0f, x.y)); };
  float2 r0, r1, r2;
  if (z) {
    const float2 d02 = __ffma2_rn(m1, t2, t0);
    const float2 tau = make_float2(fabsf(d02.x), fabsf(d02.y));
    r0 = __fmul2_rn(__fadd2_rn(t0, tau), rcp2(t0));
    r1 = __fmul2_rn(__fadd2_rn(t1, tau), rcp2(t1));
    r2 = __fmul2_rn(__fadd2_rn(t2, tau), rcp2(t2));
  } else {
    r0 = rcp2(__fmul2_rn(t0, t0));
    r1 = rcp2(__fmul2_rn(t1, t1));
    r2 = rcp2(__fmul2_rn(t2, t2));
  }
  const float2 g0 = __ffma2_rn(c(5.0f / 18.0f), D2, __fmul2_rn(c(1.0f / 9.0f), D1));
  const float2 g1 = __ffma2_rn(c(2.0f / 3.0f), D3, __fmul2_rn(c(1.0f / 3.0f), D2));
  const float2 g2 = __ffma2_rn(c(2.0f / 3.0f), D3, __fmul2_rn(c(1.0f / 6.0f), D4));
  const float2 num = __ffma2_rn(r2, g2, __ffma2_rn(r1, g1, __fmul2_rn(r0, g0)));
  const float2 den = __ffma2_rn(c(1.0f / 3.0f), r0, __ffma2_rn(c(2.0f), r1, r2));
  return __ffma2_rn(num, rcp2(den), v0);
}

// WENO5-JS per cell: both face values one cell j contributes, from the same
// five values v[j-2..j+2]:
//   right = v^-_{j+1/2} (left-biased, the weno5 formula above),
//   left  = v^+_{j-1/2} (right-biased: the same formula on the mirrored
//           stencil v[j+2..j-2]).
// The mirrored stencil has the smoothness indicators in reverse order
// (beta'_k = beta_{2-k}: the three 3-cell sub-stencils are the same), so
// both values share the indicators and their reciprocals; only the linear
// weights and candidates differ.  With the differences D1..D4 of weno5_pair
// the mirrored ones are D1' = -D4, D2' = -D3, D3' = -D2, D4' = -D1.
// Equal to two weno5 calls up to rounding.  z = 1: WENO5-Z (Table 2; alpha_k
// = d_k (1 + tau5 / (eps + beta_k)), tau5 = |beta_0 - beta_2|, the same for
// the mirrored stencil, so the two values share the weights' factors too).
template <typename T>
JF_HD void weno5_cell(T vm2, T vm1, T v0, T vp1, T vp2, T eps, T& right, T& left, int z = 0) {
  const T D1 = vm2 - vm1, D2 = v0 - vm1, D3 = vp1 - v0, D4 = vp1 - vp2;
  const T c13 = T(13) / T(12);
  const T d0 = D2 + D1, e0 = T(3) * D2 + D1;
  const T d1 = D3 - D2, e1 = D2 + D3;
  const T d2 = D3 + D4, e2 = T(3) * D3 + D4;
  const T t0 = eps + (c13 * d0 * d0 + T(0.25) * e0 * e0);
  const T t1 = eps + (c13 * d1 * d1 + T(0.25) * e1 * e1);
  const T t2 = eps + (c13 * d2 * d2 + T(0.25) * e2 * e2);
  // candidate offsets q_k - v0 (times 6) of both reconstructions
  const T g0 = T(5) * D2 + T(2) * D1, g1 = D2 + T(2) * D3, g2 = T(4) * D3 + D4;
  const T h0 = -(T(5) * D3 + T(2) * D4), h1 = -(D3 + T(2) * D2), h2 = -(T(4) * D2 + D1);
  if constexpr (sizeof(T) == 8) {
    // alpha_k scaled by the common product (t0 t1 t2)^2 (one division per
    // value; the factors are >= eps, far inside the FP64 range):
    // right: (0.1 s1 s2, 0.6 s0 s2, 0.3 s0 s1); left (mirrored t):
    // (0.1 s0 s1, 0.6 s0 s2, 0.3 s1 s2), s_k = t_k^2.  WENO5-Z: the factors
    // 1 + tau5 / t_k scaled by t0 t1 t2: u_k = (t_k + tau5) t_i t_j, the left
    // value taking them in reverse order
    T a0, a1, a2, b0, b2;
    if (z) {
      const T tau = fabs(t0 - t2);
      const T u0 = (t0 + tau) * (t1 * t2), u1 = (t1 + tau) * (t0 * t2), u2 = (t2 + tau) * (t0 * t1);
      a0 = T(0.1) * u0;
      a1 = T(0.6) * u1;
      a2 = T(0.3) * u2;
      b0 = T(0.1) * u2;
      b2 = T(0.3) * u0;
    } else {
      const T s0 = t0 * t0, s1 = t1 * t1, s2 = t2 * t2;
      const T p12 = s1 * s2, p02 = s0 * s2, p01 = s0 * s1;
      a0 = T(0.1) * p12;
      a1 = T(0.6) * p02;
      a2 = T(0.3) * p01;
      b0 = T(0.1) * p01;
      b2 = T(0.3) * p12;
    }
    // one division for both values: 1/D_r = D_l / (D_r D_l) and the converse
    // (D >= 6e-25 as every s_k >= eps^2; the product stays far inside the
    // FP64 range)
    const T Dr = T(6) * (a0 + a1 + a2), Dl = T(6) * (b0 + a1 + b2);
    const T inv = T(1) / (Dr * Dl);
    right = v0 + (a0 * g0 + a1 * g1 + a2 * g2) * (Dl * inv);
    left = v0 + (b0 * h0 + a1 * h1 + b2 * h2) * (Dr * inv);
  } else {
    T r0, r1, r2;
    if (z) {
      const T tau = fabs(t0 - t2);
      r0 = (t0 + tau) * trcp(t0);
      r1 = (t1 + tau) * trcp(t1);
      r2 = (t2 + tau) * trcp(t2);
    } else {
      r0 = trcp(t0 * t0);
      r1 = trcp(t1 * t1);
      r2 = trcp(t2 * t2);
    }
    const T a0 = T(0.1) * r0, a1 = T(0.6) * r1, a2 = T(0.3) * r2;
    const T b0 = T(0.1) * r2, b2 = T(0.3) * r0;
    right = v0 + (a0 * g0 + a1 * g1 + a2 * g2) * trcp(T(6) * (a0 + a1 + a2));
    left = v0 + (b0 * h0 + a1 * h1 + b2 * h2) * trcp(T(6) * (b0 + a1 + b2));
  }
}

// weno5_cell for two components of one cell in the lanes of packed FP32x2
// operations (the arithmetic of weno5_pair: indicators scaled by 12/13,
// linear weights scaled by 10/3; z = 1: WENO5-Z as in weno5_cell).
__device__ __forceinline__ void weno5_cell_pair(float2 vm2, float2 vm1, float2 v0, float2 vp1, float2 vp2, float eps,
                                                float2& right, float2& left, int z = 0) {
  auto c = [](float x) { return make_float2(x, x); };
  const float2 m1 = c(-1.0f);
  const float2 D1 = __ffma2_rn(m1, vm1, vm2);
  const float2 D2 = __ffma2_rn(m1, vm1, v0);
  const float2 D3 = __ffma2_rn(m1, v0, vp1);
  const float2 D4 = __ffma2_rn(m1, vp2, vp1);
  const float2 d0 = __fadd2_rn(D2, D1), e0 = __ffma2_rn(c(3.0f), D2, D1);
  const float2 d1 = __ffma2_rn(m1, D2, D3), e1 = __fadd2_rn(D2, D3);
  const float2 d2 = __fadd2_rn(D3, D4), e2 = __ffma2_rn(c(3.0f), D3, D4);
  const float2 k3 = c(3.0f / 13.0f), ke = c(12.0f / 13.0f * eps);
  const float2 t0 = __ffma2_rn(d0, d0, __ffma2_rn(__fmul2_rn(k3, e0), e0, ke));
  const float2 t1 = __ffma2_rn(d1, d1, __ffma2_rn(__fmul2_rn(k3, e1), e1, ke));
  const float2 t2 = __ffma2_rn(d2, d2, __ffma2_rn(__fmul2_rn(k3, e2), e2, ke));
  auto rcp2 = [](float2 x) { return make_float2(__fdividef(1.0f, x.x), __fdividef(1.0f, x.y)); };
  float2 r0, r1, r2;
  if (z) {
    const float2 d02 = __ffma2_rn(m1, t2, t0);
    const float2 tau = make_float2(fabsf(d02.x), fabsf(d02.y));
    r0 = __fmul2_rn(__fadd2_rn(t0, tau), rcp2(t0));
    r1 = __fmul2_rn(__fadd2_rn(t1, tau), rcp2(t1));
    r2 = __fmul2_rn(__fadd2_rn(t2, tau), rcp2(t2));
  } else {
    r0 = rcp2(__fmul2_rn(t0, t0));
    r1 = rcp2(__fmul2_rn(t1, t1));
    r2 = rcp2(__fmul2_rn(t2, t2));
  }
  // right: v0 + (r0 g0 + r1 g1 + r2 g2) / (r0/3 + 2 r1 + r2)
  const float2 g0 = __ffma2_rn(c(5.0f / 18.0f), D2, __fmul2_rn(c(1.0f / 9.0f), D1));
  const float2 g1 = __ffma2_rn(c(2.0f / 3.0f), D3, __fmul2_rn(c(1.0f / 3.0f), D2));
  const float2 g2 = __ffma2_rn(c(2.0f / 3.0f), D3, __fmul2_rn(c(1.0f / 6.0f), D4));
  const float2 num = __ffma2_rn(r2, g2, __ffma2_rn(r1, g1, __fmul2_rn(r0, g0)));
  const float2 den = __ffma2_rn(c(1.0f / 3.0f), r0, __ffma2_rn(c(2.0f), r1, r2));
  right = __ffma2_rn(num, rcp2(den), v0);
  // left: the mirrored stencil (r and D reversed and negated)
  const float2 h0 = __ffma2_rn(c(-5.0f / 18.0f), D3, __fmul2_rn(c(-1.0f / 9.0f), D4));
  const float2 h1 = __ffma2_rn(c(-2.0f / 3.0f), D2, __fmul2_rn(c(-1.0f / 3.0f), D3));
  const float2 h2 = __ffma2_rn(c(-2.0f / 3.0f), D2, __fmul2_rn(c(-1.0f / 6.0f), D1));
  const float2 numl = __ffma2_rn(r0, h2, __ffma2_rn(r1, h1, __fmul2_rn(r2, h0)));
  const float2 denl = __ffma2_rn(c(1.0f / 3.0f), r2, __ffma2_rn(c(2.0f), r1, r0));
  left = __ffma2_rn(numl, rcp2(denl), v0);
}

// WENO3-JS (Table 2): value at x_{i+1/2} biased to the left from
// v[i-1], v[i], v[i+1]: q0 = (3 v[i] - v[i-1]) / 2, q1 = (v[i] + v[i+1]) / 2,
// beta0 = (v[i] - v[i-1])^2, beta1 = (v[i+1] - v[i])^2,
// alpha_k = d_k / (eps + beta_k)^2, d = (1/3, 2/3), omega_k = alpha_k / sum.
template <typename T>
JF_HD T weno3(T vm1, T v0, T vp1, T eps) {
  const T q0 = T(0.5) * (T(3) * v0 - vm1), q1 = T(0.5) * (v0 + vp1);
  const T t0 = eps + (v0 - vm1) * (v0 - vm1), t1 = eps + (vp1 - v0) * (vp1 - v0);
  const T a0 = T(1.0 / 3.0) * trcp(t0 * t0), a1 = T(2.0 / 3.0) * trcp(t1 * t1);
  return (a0 * q0 + a1 * q1) * trcp(a0 + a1);
}
__device__ __forceinline__ float2 weno3_pair(float2 vm1, float2 v0, float2 vp1, float eps) {
  return make_float2(weno3(vm1.x, v0.x, vp1.x, eps), weno3(vm1.y, v0.y, vp1.y, eps));
}

// Signal speeds S_L <= S_R at a face along axis D (Table 2 estimates), from
// the side states W = [rho, u, v, w, p] and their total energies E, 1/rho
// and sound speeds c:
//   Einfeldt (1988): Roe averages (weights sqrt(rho)) u~, H~ (H = (E + p)/rho),
//     c~ = sqrt((gamma - 1)(H~ - |u~|^2/2)); S_L = min(u_L - c_L, u~ - c~),
//     S_R = max(u_R + c_R, u~ + c~);
//   Davis (1988): S_L = min(u_L - c_L, u_R - c_R), S_R = max(u_L + c_L, u_R + c_R);
//   Toro (1994): PVRS pressure p* = max(0, (p_L + p_R)/2 - (u_R - u_L)(rho_L + rho_R)(c_L + c_R)/8);
//     q_K = 1 if p* <= p_K else sqrt(1 + (gamma + 1)/(2 gamma)(p*/p_K - 1));
//     S_L = u_L - c_L q_L, S_R = u_R + c_R q_R.
template <typename T, int D>
JF_HD void signal_speeds(const T WL[5], const T WR[5], const Gas<T>& g, int speeds, T EL, T ER, T irL, T irR, T cL,
                         T cR, T& SL, T& SR) {
  const T rL = WL[0], rR = WR[0], pL = WL[4], pR = WR[4];
  const T unL = WL[1 + D], unR = WR[1 + D];
  if (speeds == 1) {
    SL = tmin(unL - cL, unR - cR);
    SR = tmax(unL + cL, unR + cR);
  } else if (speeds == 2) {
    const T ps = tmax(T(0), T(0.5) * (pL + pR) - T(0.125) * (unR - unL) * (rL + rR) * (cL + cR));
    const T k = (g.gamma + T(1)) * trcp(T(2) * g.gamma);
    const T qL = ps > pL ? tsqrt(T(1) + k * (ps * trcp(pL) - T(1))) : T(1);
    const T qR = ps > pR ? tsqrt(T(1) + k * (ps * trcp(pR) - T(1))) : T(1);
    SL = unL - cL * qL;
    SR = unR + cR * qR;
  } else {
    // Roe weights sqrt(rho_K) / (sqrt(rho_L) + sqrt(rho_R)) from the ratio
    // q = sqrt(rho_R / rho_L): w_L = 1 / (1 + q), w_R = q w_L
    const T q = tsqrt(rR * irL);
    const T wL = trcp(T(1) + q), wR = q * wL;
    const T HL = (EL + pL) * irL, HR = (ER + pR) * irR;
    const T u0 = wL * WL[1] + wR * WR[1];
    const T u1 = wL * WL[2] + wR * WR[2];
    const T u2 = wL * WL[3] + wR * WR[3];
    const T Ht = wL * HL + wR * HR;
    const T ct = tsqrt(g.gm1 * (Ht - T(0.5) * (u0 * u0 + u1 * u1 + u2 * u2)));
    const T un_t = D == 0 ? u0 : (D == 1 ? u1 : u2);
    SL = tmin(unL - cL, un_t - ct);
    SR = tmax(unR + cR, un_t + ct);
  }
}

// Total energy, 1/rho and sound speed of one side.
template <typename T>
JF_HD void side_state(const T W[5], const Gas<T>& g, T& E, T& ir, T& c) {
  E = W[4] * g.inv_gm1 + T(0.5) * W[0] * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
  ir = trcp(W[0]);
  c = tsqrt(g.gamma * W[4] * ir);
}

// Both sides' E, 1/rho and c; FP64 forms the two reciprocals from one
// division, 1/rho_L = rho_R / (rho_L rho_R) and the converse.
template <typename T>
JF_HD void side_states(const T WL[5], const T WR[5], const Gas<T>& g, T& EL, T& ER, T& irL, T& irR, T& cL,
                       T& cR) {
  if constexpr (sizeof(T) == 8) {
    const T inv = T(1) / (WL[0] * WR[0]);
    irL = WR[0] * inv;
    irR = WL[0] * inv;
    EL = WL[4] * g.inv_gm1 + T(0.5) * WL[0] * (WL[1] * WL[1] + WL[2] * WL[2] + WL[3] * WL[3]);
    ER = WR[4] * g.inv_gm1 + T(0.5) * WR[0] * (WR[1] * WR[1] + WR[2] * WR[2] + WR[3] * WR[3]);
    cL = tsqrt(g.gamma * WL[4] * irL);
    cR = tsqrt(g.gamma * WR[4] * irR);
  } else {
    side_state(WL, g, EL, irL, cL);
    side_state(WR, g, ER, irR, cR);
  }
}

// Physical flux along D and conservative state of one side.
template <typename T, int D>
JF_HD void side_flux(const T W[5], T E, T F[5], T U[5]) {
  const T un = W[1 + D], mass = W[0] * un;
  F[0] = mass;
  F[1] = mass * W[1];
  F[2] = mass * W[2];
  F[3] = mass * W[3];
  F[1 + D] += W[4];
  F[4] = un * (E + W[4]);
  U[0] = W[0];
  U[1] = W[0] * W[1];
  U[2] = W[0] * W[2];
  U[3] = W[0] * W[3];
  U[4] = E;
}

// HLLC flux along axis D from the reconstructed primitive states
// W = [rho, u, v, w, p] left (WL) and right (WR) of the face; `speeds` picks
// the signal speed estimate (0 Einfeldt, 1 Davis, 2 Toro).
//   U_K, F_K                conservative state and physical flux of side K
//   S_L, S_R                signal speeds of the selected estimate
//   S*  = (p_R - p_L + rho_L u_L (S_L - u_L) - rho_R u_R (S_R - u_R))
//         / (rho_L (S_L - u_L) - rho_R (S_R - u_R))
//   F*_K = F_K + S_K (U*_K - U_K),
//   U*_K = rho_K (S_K - u_K)/(S_K - S*) [1, S*, u_t, E_K/rho_K + (S* - u_K)(S* + p_K/(rho_K (S_K - u_K)))]
template <typename T, int D>
JF_HD void hllc(const T WL[5], const T WR[5], const Gas<T>& g, T F[5], int speeds = 0) {
  const T rL = WL[0], rR = WR[0], pL = WL[4], pR = WR[4];
  const T unL = WL[1 + D], unR = WR[1 + D];
  // every division goes through a reciprocal (1/rho of each side shared)
  T EL, ER, irL, irR, cL, cR;
  side_states(WL, WR, g, EL, ER, irL, irR, cL, cR);
  T SL, SR;
  signal_speeds<T, D>(WL, WR, g, speeds, EL, ER, irL, irR, cL, cR, SL, SR);
  const T mL = rL * (SL - unL), mR = rR * (SR - unR);
  const T Ss = (pR - pL + mL * unL - mR * unR) * trcp(mL - mR);
  // side selection: F_L if 0 <= S_L; F*_L if S_L < 0 <= S*; F*_R if S* < 0 < S_R; F_R if S_R <= 0
  const bool left = (SL >= T(0)) || (Ss >= T(0));
  const bool star = left ? !(SL >= T(0)) : (SR > T(0));
  const T r = left ? rL : rR, p = left ? pL : pR, un = left ? unL : unR, E = left ? EL : ER;
  const T ir = left ? irL : irR;
  const T w0 = left ? WL[1] : WR[1], w1 = left ? WL[2] : WR[2], w2 = left ? WL[3] : WR[3];
  const T S = left ? SL : SR, m = left ? mL : mR;
  // physical flux F_K of the chosen side, plus S_K (U*_K - U_K) on a star
  // side.  Mass: r u_n + S (fac - r); a tangential momentum component is
  // (r u_n + S (fac - r)) u_t on either branch (its U* - U is (fac - r) u_t),
  // so it is the mass flux times u_t; normal momentum: r u_n^2 + p +
  // S (fac S* - r u_n); energy: u_n (E + p) + S (fac e* - E).
  const T mass = r * un;
  T F0 = mass, Fn = mass * un + p, F4 = un * (E + p);
  if (star) {
    // fac = m / (S - S*) and p / m; FP64 takes both from one division,
    // x = 1 / (m (S - S*)) (m and S - S* are non-zero on a star side:
    // S_L < u_L - c_L, S_L < 0 <= S*, and the mirror image)
    T fac, p_m;
    if constexpr (sizeof(T) == 8) {
      const T d = S - Ss, x = T(1) / (m * d);
      fac = m * m * x;
      p_m = p * d * x;
    } else {
      fac = m * trcp(S - Ss);
      p_m = p * trcp(m);
    }
    F0 = mass + S * (fac - r);
    Fn = Fn + S * (fac * Ss - mass);
    F4 = F4 + S * (fac * (E * ir + (Ss - un) * (Ss + p_m)) - E);
  }
  F[0] = F0;
  F[1] = F0 * w0;
  F[2] = F0 * w1;
  F[3] = F0 * w2;
  F[1 + D] = Fn;
  F[4] = F4;
}

// HLL flux (Harten, Lax, van Leer 1983): F_L if 0 <= S_L, F_R if S_R <= 0,
// else (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L).
template <typename T, int D>
JF_HD void hll(const T WL[5], const T WR[5], const Gas<T>& g, T F[5], int speeds = 0) {
  T EL, ER, irL, irR, cL, cR;
  side_states(WL, WR, g, EL, ER, irL, irR, cL, cR);
  T SL, SR;
  signal_speeds<T, D>(WL, WR, g, speeds, EL, ER, irL, irR, cL, cR, SL, SR);
  T FL[5], FR[5], UL[5], UR[5];
  side_flux<T, D>(WL, EL, FL, UL);
  side_flux<T, D>(WR, ER, FR, UR);
  if (SL >= T(0)) {
#pragma unroll
    for (int q = 0; q < 5; ++q) F[q] = FL[q];
  } else if (SR <= T(0)) {
#pragma unroll
    for (int q = 0; q < 5; ++q) F[q] = FR[q];
  } else {
    const T inv = trcp(SR - SL);
#pragma unroll
    for (int q = 0; q < 5; ++q) F[q] = (SR * FL[q] - SL * FR[q] + SL * SR * (UR[q] - UL[q])) * inv;
  }
}

// Local Lax-Friedrichs (Rusanov): a = max(|u_L| + c_L, |u_R| + c_R),
// F = (F_L + F_R)/2 - a (U_R - U_L)/2.
template <typename T, int D>
JF_HD void rusanov(const T WL[5], const T WR[5], const Gas<T>& g, T F[5]) {
  T EL, ER, irL, irR, cL, cR;
  side_states(WL, WR, g, EL, ER, irL, irR, cL, cR);
  const T a = tmax(fabs(WL[1 + D]) + cL, fabs(WR[1 + D]) + cR);
  T FL[5], FR[5], UL[5], UR[5];
  side_flux<T, D>(WL, EL, FL, UL);
  side_flux<T, D>(WR, ER, FR, UR);
#pragma unroll
  for (int q = 0; q < 5; ++q) F[q] = T(0.5) * (FL[q] + FR[q]) - T(0.5) * a * (UR[q] - UL[q]);
}

template <typename T> JF_HD T texp(T x);
template <> JF_HD float texp<float>(float x) { return expf(x); }
template <> JF_HD double texp<double>(double x) { return exp(x); }
template <typename T> JF_HD T tlog(T x);
template <> JF_HD float tlog<float>(float x) { return logf(x); }
template <> JF_HD double tlog<double>(double x) { return log(x); }

// alpha = exp(NN(x)) of the Rusanov-NN flux; th: the network parameters.
// Not inlined: one copy of the ~2200 multiply-adds serves every face
// direction, and its 64 hidden values do not add to the register pressure
// of the tile code around the call.
#ifdef __CUDACC__
// Four consecutive network parameters (or hidden-row values) from a 16-byte
// aligned address: every weight row of the parameter layout starts at a
// multiple of 4 elements, and the kernels place the parameters at a 16-byte
// aligned offset of their shared memory.
__device__ __forceinline__ void ld4(const float* p, float o[4]) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  o[0] = q.x; o[1] = q.y; o[2] = q.z; o[3] = q.w;
}
__device__ __forceinline__ void ld4(const double* p, double o[4]) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
#endif

template <typename T>
__host__ __device__ __noinline__ T nn_alpha(const T* th, const T x[4]) {
  const T* W1 = th;
  const T* b1 = W1 + NN_HIDDEN * 4;
  const T* W2 = b1 + NN_HIDDEN;
  const T* b2 = W2 + NN_HIDDEN * NN_HIDDEN;
  const T* W3 = b2 + NN_HIDDEN;
  const T* b3 = W3 + NN_HIDDEN * NN_HIDDEN;
  const T* W4 = b3 + NN_HIDDEN;
  const T b4 = W4[NN_HIDDEN];
  T h1[NN_HIDDEN], h2[NN_HIDDEN];
#ifdef __CUDA_ARCH__
  // device: th is 16-byte aligned shared memory; weight rows read four at a time
#pragma unroll
  for (int i = 0; i < NN_HIDDEN; ++i) {
    T w[4];
    ld4(W1 + 4 * i, w);
    h1[i] = tmax(T(0), b1[i] + w[0] * x[0] + w[1] * x[1] + w[2] * x[2] + w[3] * x[3]);
  }
#pragma unroll
  for (int i = 0; i < NN_HIDDEN; ++i) {
    T z = b2[i];
#pragma unroll
    for (int j = 0; j < NN_HIDDEN; j += 4) {
      T w[4];
      ld4(W2 + NN_HIDDEN * i + j, w);
      z += w[0] * h1[j] + w[1] * h1[j + 1] + w[2] * h1[j + 2] + w[3] * h1[j + 3];
    }
    h2[i] = tmax(T(0), z);
  }
  T out = b4;
#pragma unroll 4
  for (int i = 0; i < NN_HIDDEN; ++i) {
    T z = b3[i];
#pragma unroll
    for (int j = 0; j < NN_HIDDEN; j += 4) {
      T w[4];
      ld4(W3 + NN_HIDDEN * i + j, w);
      z += w[0] * h2[j] + w[1] * h2[j + 1] + w[2] * h2[j + 2] + w[3] * h2[j + 3];
    }
    out += W4[i] * tmax(T(0), z);
  }
#else
#pragma unroll
  for (int i = 0; i < NN_HIDDEN; ++i) {
    const T z = b1[i] + W1[4 * i] * x[0] + W1[4 * i + 1] * x[1] + W1[4 * i + 2] * x[2] + W1[4 * i + 3] * x[3];
    h1[i] = tmax(T(0), z);
  }
#pragma unroll
  for (int i = 0; i < NN_HIDDEN; ++i) {
    T z = b2[i];
#pragma unroll
    for (int j = 0; j < NN_HIDDEN; ++j) z += W2[NN_HIDDEN * i + j] * h1[j];
    h2[i] = tmax(T(0), z);
  }
  T out = b4;
#pragma unroll 4
  for (int i = 0; i < NN_HIDDEN; ++i) {
    T z = b3[i];
#pragma unroll
    for (int j = 0; j < NN_HIDDEN; ++j) z += W3[NN_HIDDEN * i + j] * h2[j];
    out += W4[i] * tmax(T(0), z);
  }
#endif
  return texp(out);
}

// Network inputs of the Rusanov-NN flux at a face along D (Section 7.4):
// |u_R - u_L|, (u_L + u_R)/2, (c_L + c_R)/2, |s_R - s_L| with u the normal
// velocity and s = ln(p / rho^gamma) / (gamma - 1).
template <typename T, int D>
JF_HD void nn_inputs(const T WL[5], const T WR[5], const Gas<T>& g, T cL, T cR, T x[4]) {
  const T sL = (tlog(WL[4]) - g.gamma * tlog(WL[0])) * g.inv_gm1;
  const T sR = (tlog(WR[4]) - g.gamma * tlog(WR[0])) * g.inv_gm1;
  x[0] = fabs(WR[1 + D] - WL[1 + D]);
  x[1] = T(0.5) * (WL[1 + D] + WR[1 + D]);
  x[2] = T(0.5) * (cL + cR);
  x[3] = fabs(sR - sL);
}

// Rusanov-NN (Section 7.4, Eq. (Rusanov)): F = (F_L + F_R)/2 - alpha (U_R - U_L)/2
// with alpha = exp(NN(x)).
template <typename T, int D>
JF_HD void rusanov_nn(const T WL[5], const T WR[5], const Gas<T>& g, T F[5]) {
  T EL, ER, irL, irR, cL, cR;
  side_states(WL, WR, g, EL, ER, irL, irR, cL, cR);
  T x[4];
  nn_inputs<T, D>(WL, WR, g, cL, cR, x);
  const T a = nn_alpha(g.nn, x);
  T FL[5], FR[5], UL[5], UR[5];
  side_flux<T, D>(WL, EL, FL, UL);
  side_flux<T, D>(WR, ER, FR, UR);
#pragma unroll
  for (int q = 0; q < 5; ++q) F[q] = T(0.5) * (FL[q] + FR[q]) - T(0.5) * a * (UR[q] - UL[q]);
}

// The Riemann solver and signal speeds of the configuration (uniform branch;
// the default kernels call hllc with Einfeldt speeds directly).
template <typename T, int D>
JF_HD void riemann_flux(const T WL[5], const T WR[5], const Gas<T>& g, T F[5]) {
  if (g.flux == 1) hll<T, D>(WL, WR, g, F, g.speeds);
  else if (g.flux == 2) rusanov<T, D>(WL, WR, g, F);
  else hllc<T, D>(WL, WR, g, F, g.speeds);
}

// Section 3.4 stencils (without the 1/h factor).
template <typename T>
JF_HD T df4(T a, T b, T c, T d) {  // face derivative * h
  return (a - T(27) * b + T(27) * c - d) * (T(1) / T(24));
}
template <typename T>
JF_HD T dc4(T m2, T m1, T p1, T p2) {  // cell-centre derivative * h
  return (m2 - T(8) * m1 + T(8) * p1 - p2) * (T(1) / T(12));
}
template <typename T>
JF_HD T rc4(T a, T b, T c, T d) {  // face interpolation
  return (-a + T(9) * b + T(9) * c - d) * (T(1) / T(16));
}

}  // namespace jf

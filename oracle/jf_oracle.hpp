// The oracle: a plain, slow, obviously-correct CPU implementation of the
// finite-volume right-hand side and TVD-RK3 step of the compressible
// Euler / Navier-Stokes equations for an ideal gas, as described in
// JAX-FLUIDS (Bezgin, Buhendwa, Adams; arXiv 2203.13760).
//
// TEST INFRASTRUCTURE ONLY.  It is compiled into oracle/liboracle.so and may be
// loaded only by tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
// reference leg.  The GPU library never includes, links or calls it, and it
// shares no code with the GPU library.
//
// Everything is templated on the scalar type T:
//   * T = double : the reference result (FP64, compiled with -ffp-contract=off);
//   * T = Dual   : forward-mode derivative, giving exact JVPs of the RK3 step;
//   * T = Counted: counts the floating-point operations of the definition.
//
// Data: ghost-padded arrays with NG = 3 ghost cells on every active axis,
// filled by sequential per-axis copies (x, then y, then z).  This is a
// deliberately different mechanism from the GPU's in-kernel index maps.
//
// Steps, each in the paper's order and notation:
//   fill_ghosts        Section 3.7 / Table 2 boundary conditions (periodic,
//                      zero gradient)
//   primitives         Section 2: W = [rho, u, v, w, p] from U = [rho, rho u,
//                      rho v, rho w, E], E = rho e + rho |u|^2 / 2, Eq.
//                      (StiffenedGas) with B = 0; T = p / (rho R)
//   weno5_js           Section 3.3 "High-order Godunov approach" step 1 with
//                      WENO5-JS (Jiang & Shu 1996, cited in Section 3.1/Table 2)
//   weno5_z            WENO5-Z (Borges et al. 2008), the "Z" of Table 2's
//                      WENO5-JS/Z
//   signal_speeds      Table 2 signal speed estimates: Einfeldt (Appendix A
//                      default), Davis (1988), Toro (1994, PVRS pressure)
//   hllc_flux          Section 3.3 steps 2-3, Eq. (ApproxRiemannSolver) with
//                      HLLC (Toro 1994) and the chosen signal speeds
//   hll_flux           HLL (Harten, Lax, van Leer 1983), Table 2
//   rusanov_flux       local Lax-Friedrichs / Rusanov, Table 2
//   rusanov_nn_flux    Section 7.4 Rusanov-NN: dissipation from an MLP
//   weno3_js           Table 2 WENO3-JS (the ground-truth scheme of Section 7.4)
//   roe_eigensystem,   Section 3.3 "Flux-Splitting approach" with the Roe
//   flux_splitting_    average and Roe flux splitting: the paper's ROE setup
//   face_flux          (Section 5: WENO5 in characteristic space)
//   dissipative_flux   Section 2 (tau, q = -lambda grad T) discretised by
//                      Section 3.4 (face C4 derivative, cell-centre C4
//                      derivative + fourth-order interpolation to the face)
//   rhs                Eq. (FVD) of Section 3.1, one-point face quadrature,
//                      dimension by dimension
//   rk3_step           Section 3.2, TVD-RK3 (Gottlieb & Shu 1998), Shu-Osher form
//   time_step          Table 2 time integrators: TVD-RK3, TVD-RK2 (Gottlieb &
//                      Shu 1998, Shu-Osher form), explicit Euler
//   compute_dt         Section 3.2 CFL criterion (the paper defers the formula
//                      to another paper; the reading used is written out below)
#pragma once
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <type_traits>
#include <vector>

#include "dual.hpp"

namespace orc {

enum { BC_PERIODIC = 0, BC_ZERO_GRADIENT = 1, BC_WALL = 2 };
// scheme options of Table 2 (0 = the Appendix A configuration)
enum { FLUX_HLLC = 0, FLUX_HLL = 1, FLUX_RUSANOV = 2, FLUX_ROE_FS = 3, FLUX_RUSANOV_NN = 4 };
enum { RECON_WENO5_JS = 0, RECON_WENO5_Z = 1, RECON_WENO3_JS = 2 };
// the Rusanov-NN dissipation network (Section 7.4): 4 inputs, three hidden
// layers of 32 ReLU units, one exponential output; parameters in the order
// W1 [32][4], b1 [32], W2 [32][32], b2 [32], W3 [32][32], b3 [32], W4 [32], b4
constexpr int NN_HIDDEN = 32;
constexpr int NN_PARAMS = 32 * 4 + 32 + 2 * (32 * 32 + 32) + 32 + 1;
enum { SPEED_EINFELDT = 0, SPEED_DAVIS = 1, SPEED_TORO = 2 };
enum { TIME_RK3 = 0, TIME_RK2 = 1, TIME_EULER = 2 };
constexpr int NG = 3;  // ghost cells per side on an active axis (WENO5 reaches 3)

// Problem description.  An axis with n == 1 is inactive (no fluxes along it).
struct Config {
  int n[3];
  double lo[3], hi[3];
  int bc[6];          // x-lo, x-hi, y-lo, y-hi, z-lo, z-hi (W, E, S, N, B, T)
  double gamma, R;    // ratio of specific heats, specific gas constant
  double mu, Pr;      // dynamic viscosity, Prandtl number
  double eps;         // WENO5-JS epsilon
  double cfl;         // CFL number
  int convective;     // include the convective (WENO5 + HLLC) fluxes
  int viscous;        // include the viscous stresses
  int heat;           // include the heat flux
  int safe;           // "is_safe_reconstruction": first-order fallback at a
                      // face side whose reconstructed rho or p is <= 0
  int flux;           // FLUX_*: Riemann solver
  int recon;          // RECON_*: reconstruction
  int speeds;         // SPEED_*: signal speed estimate (HLLC, HLL)
  int integrator;     // TIME_*: time integration
  const double* nn;   // FLUX_RUSANOV_NN: the NN_PARAMS network parameters
  const double* nn_dot;  // optional tangent of the parameters (dual-number runs)
};

inline bool active(const Config& c, int d) { return c.n[d] > 1; }
inline double spacing(const Config& c, int d) { return (c.hi[d] - c.lo[d]) / c.n[d]; }
// heat conductivity from the Prandtl number: lambda = mu c_p / Pr,
// c_p = gamma R / (gamma - 1)
inline double conductivity(const Config& c) {
  return c.heat ? c.mu * c.gamma * c.R / ((c.gamma - 1.0) * c.Pr) : 0.0;
}

// ---------------------------------------------------------------------------
// Ghost-padded multi-component field.
template <class T>
struct Field {
  int n[3], g[3], s[3], ncomp;
  std::vector<T> a;
  Field(const Config& c, int ncomp_) : ncomp(ncomp_) {
    for (int d = 0; d < 3; ++d) {
      n[d] = c.n[d];
      g[d] = active(c, d) ? NG : 0;
      s[d] = n[d] + 2 * g[d];
    }
    a.assign((size_t)ncomp * s[0] * s[1] * s[2], T(0.0));
  }
  size_t index(int m, int i, int j, int k) const {
    return (((size_t)m * s[2] + (k + g[2])) * s[1] + (j + g[1])) * s[0] + (i + g[0]);
  }
  T& operator()(int m, int i, int j, int k) { return a[index(m, i, j, k)]; }
  const T& operator()(int m, int i, int j, int k) const { return a[index(m, i, j, k)]; }
};

// Cell index shifted by `off` along axis d.
struct Cell {
  int i[3];
  Cell(int a, int b, int c) { i[0] = a; i[1] = b; i[2] = c; }
  Cell shift(int d, int off) const { Cell r = *this; r.i[d] += off; return r; }
};
template <class T>
inline const T& at(const Field<T>& f, int m, const Cell& c) { return f(m, c.i[0], c.i[1], c.i[2]); }

// Boundary conditions (Section 3.7, Table 2): periodic, wall (symmetry) or zero gradient
// (the ghost cell copies the nearest interior cell; "transmissive",
// "neumann" with zero flux in Appendix A).  Axes are filled one after the
// other; each later axis copies whole ghost-extended lines of the earlier
// ones, which also fills the edge and corner ghost cells.
template <class T>
void fill_ghosts(Field<T>& f, const Config& c) {
  for (int d = 0; d < 3; ++d) {
    if (!active(c, d)) continue;
    const int n = c.n[d];
    // one visit per line along d; the other axes run over their ghost-extended
    // range if they were filled before d, else over the interior
    int lo[3], hi[3];
    for (int e = 0; e < 3; ++e) {
      if (e < d) { lo[e] = -f.g[e]; hi[e] = f.n[e] + f.g[e]; }
      else { lo[e] = 0; hi[e] = f.n[e]; }
    }
    lo[d] = 0;
    hi[d] = 1;
    for (int m = 0; m < f.ncomp; ++m)
      for (int k = lo[2]; k < hi[2]; ++k)
        for (int j = lo[1]; j < hi[1]; ++j)
          for (int i = lo[0]; i < hi[0]; ++i) {
            const Cell base(i, j, k);
            for (int q = 1; q <= NG; ++q) {
              // low-side ghost -q and high-side ghost n-1+q, with their sources
              Cell glo = base, ghi = base, slo = base, shi = base;
              glo.i[d] = -q;
              ghi.i[d] = n - 1 + q;
              // periodic: wrap; zero gradient: the nearest cell; wall: the
              // mirror cell with the normal momentum negated (slip wall)
              const int blo = c.bc[2 * d], bhi = c.bc[2 * d + 1];
              slo.i[d] = blo == BC_PERIODIC ? n - q : (blo == BC_WALL ? q - 1 : 0);
              shi.i[d] = bhi == BC_PERIODIC ? q - 1 : (bhi == BC_WALL ? n - q : n - 1);
              const double sgn_lo = (blo == BC_WALL && m == 1 + d) ? -1.0 : 1.0;
              const double sgn_hi = (bhi == BC_WALL && m == 1 + d) ? -1.0 : 1.0;
              f(m, glo.i[0], glo.i[1], glo.i[2]) = sgn_lo * f(m, slo.i[0], slo.i[1], slo.i[2]);
              f(m, ghi.i[0], ghi.i[1], ghi.i[2]) = sgn_hi * f(m, shi.i[0], shi.i[1], shi.i[2]);
            }
          }
  }
}

// ---------------------------------------------------------------------------
// Section 2: primitive variables from conservative ones; ideal gas (Eq.
// StiffenedGas with B = 0): p = (gamma - 1) (E - rho |u|^2 / 2).
// Component 5 holds the temperature T = p / (rho R) (Section 2, Fourier law).
template <class T>
void primitives(const Field<T>& U, Field<T>& W, const Config& c) {
  for (int k = -U.g[2]; k < U.n[2] + U.g[2]; ++k)
    for (int j = -U.g[1]; j < U.n[1] + U.g[1]; ++j)
      for (int i = -U.g[0]; i < U.n[0] + U.g[0]; ++i) {
        const T rho = U(0, i, j, k);
        const T u = U(1, i, j, k) / rho;
        const T v = U(2, i, j, k) / rho;
        const T w = U(3, i, j, k) / rho;
        const T kinetic = 0.5 * rho * (u * u + v * v + w * w);
        const T p = (c.gamma - 1.0) * (U(4, i, j, k) - kinetic);
        W(0, i, j, k) = rho;
        W(1, i, j, k) = u;
        W(2, i, j, k) = v;
        W(3, i, j, k) = w;
        W(4, i, j, k) = p;
        W(5, i, j, k) = p / (rho * c.R);
      }
}

template <class T> inline T sq(const T& x) { return x * x; }
// rho^gamma = exp(gamma ln rho) (rho > 0)
template <class T> inline T pow_gamma(const T& r, double gamma) { return exp(gamma * log(r)); }
template <class T> inline T tmin(const T& a, const T& b) { return (b < a) ? b : a; }
template <class T> inline T tmax(const T& a, const T& b) { return (a < b) ? b : a; }

// WENO5-JS (Jiang & Shu 1996), the reconstruction named "WENO5-JS" in Table 2
// and Appendix A.  Given cell values v[i-2], ..., v[i+2] it returns the value
// at the face x_{i+1/2} biased to the left (the state W^-_{i+1/2}).
//   q_k   third-order candidate values on the three sub-stencils
//   beta_k smoothness indicators, alpha_k = d_k / (eps + beta_k)^2,
//   d = (1/10, 6/10, 3/10), omega_k = alpha_k / sum(alpha).
template <class T>
T weno5_js(const T& vm2, const T& vm1, const T& v0, const T& vp1, const T& vp2, double eps) {
  const T q0 = (2.0 * vm2 - 7.0 * vm1 + 11.0 * v0) / 6.0;
  const T q1 = (-vm1 + 5.0 * v0 + 2.0 * vp1) / 6.0;
  const T q2 = (2.0 * v0 + 5.0 * vp1 - vp2) / 6.0;
  const T b0 = (13.0 / 12.0) * sq(vm2 - 2.0 * vm1 + v0) + 0.25 * sq(vm2 - 4.0 * vm1 + 3.0 * v0);
  const T b1 = (13.0 / 12.0) * sq(vm1 - 2.0 * v0 + vp1) + 0.25 * sq(vm1 - vp1);
  const T b2 = (13.0 / 12.0) * sq(v0 - 2.0 * vp1 + vp2) + 0.25 * sq(3.0 * v0 - 4.0 * vp1 + vp2);
  const T a0 = 0.1 / sq(eps + b0);
  const T a1 = 0.6 / sq(eps + b1);
  const T a2 = 0.3 / sq(eps + b2);
  const T s = a0 + a1 + a2;
  const T w0 = a0 / s, w1 = a1 / s, w2 = a2 / s;
  return w0 * q0 + w1 * q1 + w2 * q2;
}

// WENO5-Z (Borges, Carmona, Costa, Don 2008): the candidates q_k and
// smoothness indicators beta_k of WENO5-JS, the global indicator
// tau5 = |beta_0 - beta_2| and alpha_k = d_k (1 + tau5 / (eps + beta_k)),
// omega_k = alpha_k / sum(alpha) (power 1 of the ratio).
template <class T>
T weno5_z(const T& vm2, const T& vm1, const T& v0, const T& vp1, const T& vp2, double eps) {
  const T q0 = (2.0 * vm2 - 7.0 * vm1 + 11.0 * v0) / 6.0;
  const T q1 = (-vm1 + 5.0 * v0 + 2.0 * vp1) / 6.0;
  const T q2 = (2.0 * v0 + 5.0 * vp1 - vp2) / 6.0;
  const T b0 = (13.0 / 12.0) * sq(vm2 - 2.0 * vm1 + v0) + 0.25 * sq(vm2 - 4.0 * vm1 + 3.0 * v0);
  const T b1 = (13.0 / 12.0) * sq(vm1 - 2.0 * v0 + vp1) + 0.25 * sq(vm1 - vp1);
  const T b2 = (13.0 / 12.0) * sq(v0 - 2.0 * vp1 + vp2) + 0.25 * sq(3.0 * v0 - 4.0 * vp1 + vp2);
  const T tau5 = fabs(b0 - b2);
  const T a0 = 0.1 * (1.0 + tau5 / (eps + b0));
  const T a1 = 0.6 * (1.0 + tau5 / (eps + b1));
  const T a2 = 0.3 * (1.0 + tau5 / (eps + b2));
  const T s = a0 + a1 + a2;
  const T w0 = a0 / s, w1 = a1 / s, w2 = a2 / s;
  return w0 * q0 + w1 * q1 + w2 * q2;
}

// WENO3-JS (Jiang & Shu 1996; Table 2 "WENO3-JS"): value at x_{i+1/2} biased
// to the left from v[i-1], v[i], v[i+1]: candidates q0 = (-v[i-1] + 3 v[i]) / 2,
// q1 = (v[i] + v[i+1]) / 2, smoothness beta0 = (v[i] - v[i-1])^2,
// beta1 = (v[i+1] - v[i])^2, alpha_k = d_k / (eps + beta_k)^2 with
// d = (1/3, 2/3), omega_k = alpha_k / sum(alpha).
template <class T>
T weno3_js(const T& vm1, const T& v0, const T& vp1, double eps) {
  const T q0 = (-vm1 + 3.0 * v0) / 2.0;
  const T q1 = (v0 + vp1) / 2.0;
  const T b0 = sq(v0 - vm1), b1 = sq(vp1 - v0);
  const T a0 = (1.0 / 3.0) / sq(eps + b0);
  const T a1 = (2.0 / 3.0) / sq(eps + b1);
  const T s = a0 + a1;
  return (a0 / s) * q0 + (a1 / s) * q1;
}

// Conservative state and physical flux along axis d (Section 2: F, G, H).
template <class T>
void conservative_of(const T W[5], double gamma, T U[5]) {
  U[0] = W[0];
  U[1] = W[0] * W[1];
  U[2] = W[0] * W[2];
  U[3] = W[0] * W[3];
  U[4] = W[4] / (gamma - 1.0) + 0.5 * W[0] * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
}
template <class T>
void physical_flux(const T W[5], const T U[5], int d, T F[5]) {
  const T un = W[1 + d];
  F[0] = U[0] * un;
  F[1] = U[1] * un;
  F[2] = U[2] * un;
  F[3] = U[3] * un;
  F[1 + d] = F[1 + d] + W[4];
  F[4] = un * (U[4] + W[4]);
}

// Signal speed estimates S_L <= S_R of the Riemann fan at a face with normal
// axis d (Table 2), from the side states W = [rho, u, v, w, p]:
//   Einfeldt (1988): Roe averages with weights sqrt(rho): u~, H~
//     (H = (E + p) / rho), c~ = sqrt((gamma - 1)(H~ - |u~|^2 / 2));
//     S_L = min(u_L - c_L, u~ - c~), S_R = max(u_R + c_R, u~ + c~);
//   Davis (1988): S_L = min(u_L - c_L, u_R - c_R), S_R = max(u_L + c_L, u_R + c_R);
//   Toro (1994; Toro 2009, Section 10.5.2): the primitive-variable (PVRS)
//     pressure p* = max(0, (p_L + p_R) / 2 - (u_R - u_L) rho_ c_ / 2) with
//     rho_ = (rho_L + rho_R) / 2, c_ = (c_L + c_R) / 2; per side
//     q_K = 1 if p* <= p_K, else sqrt(1 + (gamma + 1) / (2 gamma) (p* / p_K - 1));
//     S_L = u_L - c_L q_L, S_R = u_R + c_R q_R.
template <class T>
T toro_q(const T& p_star, const T& pK, double gamma) {
  if (p_star <= pK) return T(1.0);
  return sqrt(1.0 + (gamma + 1.0) / (2.0 * gamma) * (p_star / pK - 1.0));
}
// EL, ER: total energies of the two sides (already formed by the callers).
template <class T>
void signal_speeds(const T WL[5], const T WR[5], const T& EL, const T& ER, int d, double gamma, int kind, T& SL,
                   T& SR) {
  const T rhoL = WL[0], rhoR = WR[0], pL = WL[4], pR = WR[4];
  const T unL = WL[1 + d], unR = WR[1 + d];
  const T cL = sqrt(gamma * pL / rhoL);
  const T cR = sqrt(gamma * pR / rhoR);
  if (kind == SPEED_DAVIS) {
    SL = tmin(unL - cL, unR - cR);
    SR = tmax(unL + cL, unR + cR);
  } else if (kind == SPEED_TORO) {
    const T ppv = 0.5 * (pL + pR) - 0.5 * (unR - unL) * (0.5 * (rhoL + rhoR)) * (0.5 * (cL + cR));
    const T p_star = tmax(T(0.0), ppv);
    SL = unL - cL * toro_q(p_star, pL, gamma);
    SR = unR + cR * toro_q(p_star, pR, gamma);
  } else {
    const T HL = (EL + pL) / rhoL;
    const T HR = (ER + pR) / rhoR;
    const T sL = sqrt(rhoL), sR = sqrt(rhoR);
    T ut[3];
    for (int m = 0; m < 3; ++m) ut[m] = (sL * WL[1 + m] + sR * WR[1 + m]) / (sL + sR);
    const T Ht = (sL * HL + sR * HR) / (sL + sR);
    const T ct = sqrt((gamma - 1.0) * (Ht - 0.5 * (ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2])));
    SL = tmin(unL - cL, ut[d] - ct);
    SR = tmax(unR + cR, ut[d] + ct);
  }
}

// HLLC flux (Toro 1994), normal axis d, signal speeds of the chosen kind.
// Section 3.3, Eq. (ApproxRiemannSolver): F(U^-, U^+, W^-, W^+).
//   S* = (p_R - p_L + rho_L u_L (S_L - u_L) - rho_R u_R (S_R - u_R))
//        / (rho_L (S_L - u_L) - rho_R (S_R - u_R));
//   U*_K = rho_K (S_K - u_K)/(S_K - S*) [1, S* (normal), tangential u,
//          E_K/rho_K + (S* - u_K)(S* + p_K / (rho_K (S_K - u_K)))];
//   F*_K = F_K + S_K (U*_K - U_K);
//   F = F_L if 0 <= S_L; F*_L if S_L < 0 <= S*; F*_R if S* < 0 < S_R;
//       F_R if S_R <= 0.
template <class T>
void hllc_flux(const T WL[5], const T WR[5], int d, double gamma, T F[5], int speeds = SPEED_EINFELDT) {
  T UL[5], UR[5], FL[5], FR[5];
  conservative_of(WL, gamma, UL);
  conservative_of(WR, gamma, UR);
  physical_flux(WL, UL, d, FL);
  physical_flux(WR, UR, d, FR);
  const T rhoL = WL[0], rhoR = WR[0], pL = WL[4], pR = WR[4];
  const T unL = WL[1 + d], unR = WR[1 + d];
  T SL, SR;
  signal_speeds(WL, WR, UL[4], UR[4], d, gamma, speeds, SL, SR);
  const T Ss = (pR - pL + rhoL * unL * (SL - unL) - rhoR * unR * (SR - unR)) /
               (rhoL * (SL - unL) - rhoR * (SR - unR));
  if (SL >= 0.0) {
    for (int m = 0; m < 5; ++m) F[m] = FL[m];
  } else if (Ss >= 0.0) {
    const T fac = rhoL * (SL - unL) / (SL - Ss);
    T Us[5];
    Us[0] = fac;
    for (int m = 0; m < 3; ++m) Us[1 + m] = fac * WL[1 + m];
    Us[1 + d] = fac * Ss;
    Us[4] = fac * (UL[4] / rhoL + (Ss - unL) * (Ss + pL / (rhoL * (SL - unL))));
    for (int m = 0; m < 5; ++m) F[m] = FL[m] + SL * (Us[m] - UL[m]);
  } else if (SR > 0.0) {
    const T fac = rhoR * (SR - unR) / (SR - Ss);
    T Us[5];
    Us[0] = fac;
    for (int m = 0; m < 3; ++m) Us[1 + m] = fac * WR[1 + m];
    Us[1 + d] = fac * Ss;
    Us[4] = fac * (UR[4] / rhoR + (Ss - unR) * (Ss + pR / (rhoR * (SR - unR))));
    for (int m = 0; m < 5; ++m) F[m] = FR[m] + SR * (Us[m] - UR[m]);
  } else {
    for (int m = 0; m < 5; ++m) F[m] = FR[m];
  }
}

// HLL flux (Harten, Lax, van Leer 1983) for given signal speeds S_L <= S_R:
//   F = F_L if 0 <= S_L; F_R if S_R <= 0; otherwise
//   F = (S_R F_L - S_L F_R + S_L S_R (U_R - U_L)) / (S_R - S_L).
template <class T>
void hll_flux_speeds(const T WL[5], const T WR[5], int d, double gamma, const T& SL, const T& SR, T F[5]) {
  T UL[5], UR[5], FL[5], FR[5];
  conservative_of(WL, gamma, UL);
  conservative_of(WR, gamma, UR);
  physical_flux(WL, UL, d, FL);
  physical_flux(WR, UR, d, FR);
  if (SL >= 0.0) {
    for (int m = 0; m < 5; ++m) F[m] = FL[m];
  } else if (SR <= 0.0) {
    for (int m = 0; m < 5; ++m) F[m] = FR[m];
  } else {
    for (int m = 0; m < 5; ++m) F[m] = (SR * FL[m] - SL * FR[m] + SL * SR * (UR[m] - UL[m])) / (SR - SL);
  }
}
template <class T>
void hll_flux(const T WL[5], const T WR[5], int d, double gamma, T F[5], int speeds = SPEED_EINFELDT) {
  T UL[5], UR[5];
  conservative_of(WL, gamma, UL);
  conservative_of(WR, gamma, UR);
  T SL, SR;
  signal_speeds(WL, WR, UL[4], UR[4], d, gamma, speeds, SL, SR);
  hll_flux_speeds(WL, WR, d, gamma, SL, SR, F);
}

// Local Lax-Friedrichs (Rusanov) flux: with a = max(|u_L| + c_L, |u_R| + c_R)
// (normal velocities),  F = (F_L + F_R) / 2 - a (U_R - U_L) / 2.
template <class T>
void rusanov_flux(const T WL[5], const T WR[5], int d, double gamma, T F[5]) {
  T UL[5], UR[5], FL[5], FR[5];
  conservative_of(WL, gamma, UL);
  conservative_of(WR, gamma, UR);
  physical_flux(WL, UL, d, FL);
  physical_flux(WR, UR, d, FR);
  const T cL = sqrt(gamma * WL[4] / WL[0]);
  const T cR = sqrt(gamma * WR[4] / WR[0]);
  const T a = tmax(fabs(WL[1 + d]) + cL, fabs(WR[1 + d]) + cR);
  for (int m = 0; m < 5; ++m) F[m] = 0.5 * (FL[m] + FR[m]) - 0.5 * a * (UR[m] - UL[m]);
}

// Rusanov-NN (Section 7.4, Eq. (Rusanov)): the Rusanov flux with the
// dissipation alpha given by a multi-layer perceptron of the face states,
//   F = (F_L + F_R) / 2 - alpha (U_R - U_L) / 2,
//   alpha = exp(W4 h3 + b4), h_l = ReLU(W_l h_{l-1} + b_l), h0 = x,
//   x = (|u_R - u_L|, (u_L + u_R) / 2, (c_L + c_R) / 2, |s_R - s_L|),
// with u the face-normal velocity and s = ln(p / rho^gamma) / (gamma - 1) the
// entropy (R = 1).  P is the parameter type (double, or Dual for derivatives
// with respect to the parameters).
template <class T, class P>
T nn_alpha(const P* theta, const T x[4]) {
  const P* W1 = theta;
  const P* b1 = W1 + NN_HIDDEN * 4;
  const P* W2 = b1 + NN_HIDDEN;
  const P* b2 = W2 + NN_HIDDEN * NN_HIDDEN;
  const P* W3 = b2 + NN_HIDDEN;
  const P* b3 = W3 + NN_HIDDEN * NN_HIDDEN;
  const P* W4 = b3 + NN_HIDDEN;
  const P* b4 = W4 + NN_HIDDEN;
  T h1[NN_HIDDEN], h2[NN_HIDDEN], h3[NN_HIDDEN];
  for (int i = 0; i < NN_HIDDEN; ++i) {
    T z = T(0.0) + b1[i];
    for (int j = 0; j < 4; ++j) z = z + W1[4 * i + j] * x[j];
    h1[i] = tmax(T(0.0), z);
  }
  for (int i = 0; i < NN_HIDDEN; ++i) {
    T z = T(0.0) + b2[i];
    for (int j = 0; j < NN_HIDDEN; ++j) z = z + W2[NN_HIDDEN * i + j] * h1[j];
    h2[i] = tmax(T(0.0), z);
  }
  for (int i = 0; i < NN_HIDDEN; ++i) {
    T z = T(0.0) + b3[i];
    for (int j = 0; j < NN_HIDDEN; ++j) z = z + W3[NN_HIDDEN * i + j] * h2[j];
    h3[i] = tmax(T(0.0), z);
  }
  T z = T(0.0) + b4[0];
  for (int j = 0; j < NN_HIDDEN; ++j) z = z + W4[j] * h3[j];
  return exp(z);
}
template <class T>
void rusanov_nn_flux(const Config& c, const T WL[5], const T WR[5], int d, T F[5]) {
  T UL[5], UR[5], FL[5], FR[5];
  conservative_of(WL, c.gamma, UL);
  conservative_of(WR, c.gamma, UR);
  physical_flux(WL, UL, d, FL);
  physical_flux(WR, UR, d, FR);
  const T cL = sqrt(c.gamma * WL[4] / WL[0]);
  const T cR = sqrt(c.gamma * WR[4] / WR[0]);
  const T sL = log(WL[4] / pow_gamma(WL[0], c.gamma)) / (c.gamma - 1.0);
  const T sR = log(WR[4] / pow_gamma(WR[0], c.gamma)) / (c.gamma - 1.0);
  const T x[4] = {fabs(WR[1 + d] - WL[1 + d]), 0.5 * (WL[1 + d] + WR[1 + d]), 0.5 * (cL + cR), fabs(sR - sL)};
  T alpha;
  if constexpr (std::is_same<T, Dual>::value) {
    if (c.nn_dot) {
      Dual th[NN_PARAMS];
      for (int i = 0; i < NN_PARAMS; ++i) th[i] = Dual(c.nn[i], c.nn_dot[i]);
      alpha = nn_alpha(th, x);
    } else {
      alpha = nn_alpha(c.nn, x);
    }
  } else {
    alpha = nn_alpha(c.nn, x);
  }
  for (int m = 0; m < 5; ++m) F[m] = 0.5 * (FL[m] + FR[m]) - 0.5 * alpha * (UR[m] - UL[m]);
}

// The Riemann solver of the configuration.
template <class T>
void riemann_flux(const Config& c, const T WL[5], const T WR[5], int d, T F[5]) {
  if (c.flux == FLUX_HLL) hll_flux(WL, WR, d, c.gamma, F, c.speeds);
  else if (c.flux == FLUX_RUSANOV) rusanov_flux(WL, WR, d, c.gamma, F);
  else if (c.flux == FLUX_RUSANOV_NN) rusanov_nn_flux(c, WL, WR, d, F);
  else hllc_flux(WL, WR, d, c.gamma, F, c.speeds);
}

// Roe average and eigen-decomposition of the flux Jacobian along d (Section
// 3.3, Flux-Splitting approach, steps 1-2), from the primitive states of the
// two cells beside the face:
//   sqrt(rho) weights: u~ (3 components), H~ = weighted (E + p) / rho,
//   c~ = sqrt((gamma - 1)(H~ - |u~|^2 / 2));
//   eigenvalues (u_n - c, u_n, u_t1, u_t2 ... ) = (u_n - c, u_n, u_n, u_n, u_n + c);
//   right eigenvectors (columns of R, conservative variables [rho, m, E] with
//   the normal momentum in slot 1 + d):
//     r0 = [1, u - c n, H - u_n c],  r1 = [1, u, |u|^2 / 2],
//     r2 = [0, t1, u_t1],  r3 = [0, t2, u_t2],  r4 = [1, u + c n, H + u_n c]
//   with n the unit normal and t1, t2 the two other unit axes;
//   left eigenvectors L = R^{-1} (rows), written out with
//   b1 = (gamma - 1) / c^2, b2 = b1 |u|^2 / 2:
//     l0 = 1/2 [b2 + u_n / c, -b1 u - n / c, b1],
//     l1 = [1 - b2, b1 u, -b1],
//     l2 = [-u_t1, t1, 0],  l3 = [-u_t2, t2, 0],
//     l4 = 1/2 [b2 - u_n / c, -b1 u + n / c, b1].
template <class T>
struct Eigensystem {
  T lambda[5];
  T R[5][5];  // R[row][column]
  T L[5][5];  // L[row][column] = R^{-1}
};
template <class T>
Eigensystem<T> roe_eigensystem(const T WL[5], const T WR[5], int d, double gamma) {
  T UL[5], UR[5];
  conservative_of(WL, gamma, UL);
  conservative_of(WR, gamma, UR);
  const T sL = sqrt(WL[0]), sR = sqrt(WR[0]);
  T u[3];
  for (int m = 0; m < 3; ++m) u[m] = (sL * WL[1 + m] + sR * WR[1 + m]) / (sL + sR);
  const T H = (sL * (UL[4] + WL[4]) / WL[0] + sR * (UR[4] + WR[4]) / WR[0]) / (sL + sR);
  const T q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const T c = sqrt((gamma - 1.0) * (H - 0.5 * q2));
  const int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
  Eigensystem<T> es;
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) es.R[i][j] = es.L[i][j] = T(0.0);
  const T un = u[d];
  es.lambda[0] = un - c;
  es.lambda[1] = un;
  es.lambda[2] = un;
  es.lambda[3] = un;
  es.lambda[4] = un + c;
  // right eigenvectors (columns)
  es.R[0][0] = T(1.0);
  es.R[0][1] = T(1.0);
  es.R[0][4] = T(1.0);
  for (int m = 0; m < 3; ++m) {
    es.R[1 + m][0] = u[m];
    es.R[1 + m][1] = u[m];
    es.R[1 + m][4] = u[m];
  }
  es.R[1 + d][0] = un - c;
  es.R[1 + d][4] = un + c;
  es.R[4][0] = H - un * c;
  es.R[4][1] = 0.5 * q2;
  es.R[4][4] = H + un * c;
  es.R[1 + t1][2] = T(1.0);
  es.R[4][2] = u[t1];
  es.R[1 + t2][3] = T(1.0);
  es.R[4][3] = u[t2];
  // left eigenvectors (rows)
  const T b1 = (gamma - 1.0) / (c * c);
  const T b2 = 0.5 * b1 * q2;
  es.L[0][0] = 0.5 * (b2 + un / c);
  es.L[4][0] = 0.5 * (b2 - un / c);
  es.L[1][0] = 1.0 - b2;
  for (int m = 0; m < 3; ++m) {
    es.L[0][1 + m] = -0.5 * b1 * u[m];
    es.L[4][1 + m] = -0.5 * b1 * u[m];
    es.L[1][1 + m] = b1 * u[m];
  }
  es.L[0][1 + d] = es.L[0][1 + d] - 0.5 / c;
  es.L[4][1 + d] = es.L[4][1 + d] + 0.5 / c;
  es.L[0][4] = 0.5 * b1;
  es.L[4][4] = 0.5 * b1;
  es.L[1][4] = -b1;
  es.L[2][0] = -u[t1];
  es.L[2][1 + t1] = T(1.0);
  es.L[3][0] = -u[t2];
  es.L[3][1 + t2] = T(1.0);
  return es;
}

// Flux-splitting face flux (Section 3.3, steps 3-7) with Roe flux splitting
// (Lambda_bar = |Lambda| of the Roe eigensystem): for the stencil cells
// j = i-2 .. i+3 of the face x_{i+1/2},
//   V_j = L U_j, G_j = L F_j, G^+-_j = (G_j +- |Lambda| V_j) / 2;
// G^+ at the face by the left-biased WENO5 of cells i-2..i+2, G^- by the
// mirrored stencil i+3..i-1; F = R (G^+ + G^-).
template <class T>
void flux_splitting_face_flux(const Field<T>& W, const Config& c, int d, const Cell& cell, T F[5]) {
  T Ws[6][5];
  for (int j = 0; j < 6; ++j)
    for (int m = 0; m < 5; ++m) Ws[j][m] = at(W, m, cell.shift(d, j - 2));
  const Eigensystem<T> es = roe_eigensystem(Ws[2], Ws[3], d, c.gamma);
  T Gp[6][5], Gm[6][5];
  for (int j = 0; j < 6; ++j) {
    T U[5], Fj[5];
    conservative_of(Ws[j], c.gamma, U);
    physical_flux(Ws[j], U, d, Fj);
    for (int k = 0; k < 5; ++k) {
      T v = T(0.0), g = T(0.0);
      for (int m = 0; m < 5; ++m) {
        v = v + es.L[k][m] * U[m];
        g = g + es.L[k][m] * Fj[m];
      }
      const T a = fabs(es.lambda[k]);
      Gp[j][k] = 0.5 * (g + a * v);
      Gm[j][k] = 0.5 * (g - a * v);
    }
  }
  T Gh[5];
  for (int k = 0; k < 5; ++k) {
    T gp, gm;
    if (c.recon == RECON_WENO5_Z) {
      gp = weno5_z(Gp[0][k], Gp[1][k], Gp[2][k], Gp[3][k], Gp[4][k], c.eps);
      gm = weno5_z(Gm[5][k], Gm[4][k], Gm[3][k], Gm[2][k], Gm[1][k], c.eps);
    } else if (c.recon == RECON_WENO3_JS) {
      gp = weno3_js(Gp[1][k], Gp[2][k], Gp[3][k], c.eps);
      gm = weno3_js(Gm[4][k], Gm[3][k], Gm[2][k], c.eps);
    } else {
      gp = weno5_js(Gp[0][k], Gp[1][k], Gp[2][k], Gp[3][k], Gp[4][k], c.eps);
      gm = weno5_js(Gm[5][k], Gm[4][k], Gm[3][k], Gm[2][k], Gm[1][k], c.eps);
    }
    Gh[k] = gp + gm;
  }
  for (int m = 0; m < 5; ++m) {
    T f = T(0.0);
    for (int k = 0; k < 5; ++k) f = f + es.R[m][k] * Gh[k];
    F[m] = f;
  }
}

// Convective flux at the face between cell c and cell c + e_d (Section 3.3,
// High-order Godunov approach): WENO5-JS (or -Z) on each primitive component
// in physical space ("reconstruction_var": "PRIMITIVE"), the right state by
// the mirrored stencil, then the Riemann solver (HLLC by default).
template <class T>
void convective_face_flux(const Field<T>& W, const Config& c, int d, const Cell& cell, T F[5]) {
  if (c.flux == FLUX_ROE_FS) {
    flux_splitting_face_flux(W, c, d, cell, F);
    return;
  }
  T Wm[5], Wp[5];
  for (int m = 0; m < 5; ++m) {
    const T a = at(W, m, cell.shift(d, -2));
    const T b = at(W, m, cell.shift(d, -1));
    const T e0 = at(W, m, cell);
    const T f1 = at(W, m, cell.shift(d, 1));
    const T g2 = at(W, m, cell.shift(d, 2));
    const T h3 = at(W, m, cell.shift(d, 3));
    if (c.recon == RECON_WENO5_Z) {
      Wm[m] = weno5_z(a, b, e0, f1, g2, c.eps);
      Wp[m] = weno5_z(h3, g2, f1, e0, b, c.eps);
    } else if (c.recon == RECON_WENO3_JS) {
      Wm[m] = weno3_js(b, e0, f1, c.eps);
      Wp[m] = weno3_js(g2, f1, e0, c.eps);
    } else {
      Wm[m] = weno5_js(a, b, e0, f1, g2, c.eps);
      Wp[m] = weno5_js(h3, g2, f1, e0, b, c.eps);
    }
  }
  if (c.safe) {
    // reading of "is_safe_reconstruction": if the reconstructed density or
    // pressure of a side is not positive, that side takes its cell value.
    if (!(Wm[0] > 0.0) || !(Wm[4] > 0.0))
      for (int m = 0; m < 5; ++m) Wm[m] = at(W, m, cell);
    if (!(Wp[0] > 0.0) || !(Wp[4] > 0.0))
      for (int m = 0; m < 5; ++m) Wp[m] = at(W, m, cell.shift(d, 1));
  }
  riemann_flux(c, Wm, Wp, d, F);
}

// Section 3.4 stencils.
// Face-normal fourth-order derivative at x_{i+1/2} from psi_{i-1..i+2}.
template <class T>
inline T df4(const T& a, const T& b, const T& e, const T& f, double h) {
  return (a - 27.0 * b + 27.0 * e - f) / (24.0 * h);
}
// Cell-centre fourth-order derivative at x_i from psi_{i-2}, psi_{i-1}, psi_{i+1}, psi_{i+2}.
template <class T>
inline T dc4(const T& m2, const T& m1, const T& p1, const T& p2, double h) {
  return (m2 - 8.0 * m1 + 8.0 * p1 - p2) / (12.0 * h);
}
// Fourth-order central interpolation of cell values psi_{i-1..i+2} to x_{i+1/2}.
// (The paper prints the indices i-2, i-1, i+1, i+2 for the face i+1/2; the
// symmetric stencil around the face, used here, is the reading.)
template <class T>
inline T rc4(const T& a, const T& b, const T& e, const T& f) {
  return (-a + 9.0 * b + 9.0 * e - f) / 16.0;
}

// Dissipative flux (Section 2: F^d = [0, tau^{d1}, tau^{d2}, tau^{d3},
// sum_i u_i tau^{di} - q_d], tau^{ij} = mu (du_i/dx_j + du_j/dx_i)
// - 2/3 mu delta_ij du_k/dx_k, q = -lambda grad T) at the face between cell
// c and c + e_d, discretised as in Section 3.4: derivatives along d by the
// face C4 stencil; derivatives along a tangential axis e by the cell-centre C4
// stencil at cells c-1..c+2 followed by fourth-order interpolation to the
// face; face velocities by fourth-order interpolation ("RC4", Appendix A).
template <class T>
void dissipative_face_flux(const Field<T>& W, const Config& c, int d, const Cell& cell, T Fd[5]) {
  const double hd = spacing(c, d);
  const double mu = c.viscous ? c.mu : 0.0;
  const double lambda = conductivity(c);
  // G[a][b] = du_a/dx_b at the face (only the entries tau^{d.} needs)
  T G[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) G[a][b] = T(0.0);
  Cell s[4] = {cell.shift(d, -1), cell, cell.shift(d, 1), cell.shift(d, 2)};
  for (int a = 0; a < 3; ++a)
    G[a][d] = df4(at(W, 1 + a, s[0]), at(W, 1 + a, s[1]), at(W, 1 + a, s[2]), at(W, 1 + a, s[3]), hd);
  const T dTdn = df4(at(W, 5, s[0]), at(W, 5, s[1]), at(W, 5, s[2]), at(W, 5, s[3]), hd);
  for (int e = 0; e < 3; ++e) {
    if (e == d || !active(c, e)) continue;
    const double he = spacing(c, e);
    // du_d/dx_e and du_e/dx_e are the tangential derivatives tau^{d.} uses
    const int comps[2] = {d, e};
    for (int t = 0; t < 2; ++t) {
      const int a = comps[t];
      T centre[4];
      for (int q = 0; q < 4; ++q)
        centre[q] = dc4(at(W, 1 + a, s[q].shift(e, -2)), at(W, 1 + a, s[q].shift(e, -1)),
                        at(W, 1 + a, s[q].shift(e, 1)), at(W, 1 + a, s[q].shift(e, 2)), he);
      G[a][e] = rc4(centre[0], centre[1], centre[2], centre[3]);
    }
  }
  T uf[3];
  for (int a = 0; a < 3; ++a)
    uf[a] = rc4(at(W, 1 + a, s[0]), at(W, 1 + a, s[1]), at(W, 1 + a, s[2]), at(W, 1 + a, s[3]));
  const T div = G[0][0] + G[1][1] + G[2][2];
  T tau[3];
  for (int a = 0; a < 3; ++a) {
    tau[a] = mu * (G[d][a] + G[a][d]);
    if (a == d) tau[a] = tau[a] - (2.0 / 3.0) * mu * div;
  }
  Fd[0] = T(0.0);
  Fd[1] = tau[0];
  Fd[2] = tau[1];
  Fd[3] = tau[2];
  Fd[4] = uf[0] * tau[0] + uf[1] * tau[1] + uf[2] * tau[2] + lambda * dTdn;
}

// Copy an interior SoA array U[5][nz][ny][nx] into a padded field and fill ghosts.
template <class T, class S>
void load_state(const Config& c, const S* U, Field<T>& f) {
  const size_t N = (size_t)c.n[0] * c.n[1] * c.n[2];
  for (int m = 0; m < 5; ++m)
    for (int k = 0; k < c.n[2]; ++k)
      for (int j = 0; j < c.n[1]; ++j)
        for (int i = 0; i < c.n[0]; ++i)
          f(m, i, j, k) = T(U[m * N + ((size_t)k * c.n[1] + j) * c.n[0] + i]);
  fill_ghosts(f, c);
}

// Eq. (FVD): dU/dt = - sum_d (F_{d,+} - F_{d,-}) / dx_d + sum_d (F^d_{d,+} - F^d_{d,-}) / dx_d.
// U's ghosts must be filled.  Each face flux is evaluated once (one-point Gauss
// quadrature on the face, Section 3.1) and stored; the cell then takes the
// difference of its two faces, axis by axis (dimension by dimension).
template <class T>
void rhs(const Config& c, const Field<T>& U, Field<T>& dUdt) {
  Field<T> W(c, 6);
  primitives(U, W, c);
  for (size_t q = 0; q < dUdt.a.size(); ++q) dUdt.a[q] = T(0.0);
  const bool dissipative = (c.viscous || c.heat) && c.mu != 0.0;
  for (int d = 0; d < 3; ++d) {
    if (!active(c, d)) continue;
    const double h = spacing(c, d);
    // net face flux NF = F^d - F on faces f = 0..n_d along d; face f lies
    // between cells f-1 and f
    int nf[3] = {c.n[0], c.n[1], c.n[2]};
    nf[d] += 1;
    std::vector<T> NF((size_t)5 * nf[0] * nf[1] * nf[2], T(0.0));
    const auto fidx = [&](int m, int i, int j, int k) {
      return (((size_t)m * nf[2] + k) * nf[1] + j) * nf[0] + i;
    };
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < nf[2]; ++k)
      for (int j = 0; j < nf[1]; ++j)
        for (int i = 0; i < nf[0]; ++i) {
          const Cell left = Cell(i, j, k).shift(d, -1);
          T F[5] = {T(0.0), T(0.0), T(0.0), T(0.0), T(0.0)};
          T Fd[5] = {T(0.0), T(0.0), T(0.0), T(0.0), T(0.0)};
          if (c.convective) convective_face_flux(W, c, d, left, F);
          if (dissipative) dissipative_face_flux(W, c, d, left, Fd);
          for (int m = 0; m < 5; ++m) NF[fidx(m, i, j, k)] = Fd[m] - F[m];
        }
    int e[3] = {0, 0, 0};
    e[d] = 1;
#pragma omp parallel for collapse(2) schedule(static)
    for (int k = 0; k < c.n[2]; ++k)
      for (int j = 0; j < c.n[1]; ++j)
        for (int i = 0; i < c.n[0]; ++i)
          for (int m = 0; m < 5; ++m)
            dUdt(m, i, j, k) += (NF[fidx(m, i + e[0], j + e[1], k + e[2])] - NF[fidx(m, i, j, k)]) / h;
  }
}

// Section 3.2: TVD-RK3 (Gottlieb & Shu 1998) in Shu-Osher form with fixed dt:
//   U1 = Un + dt L(Un)
//   U2 = 3/4 Un + 1/4 (U1 + dt L(U1))
//   U^{n+1} = 1/3 Un + 2/3 (U2 + dt L(U2))
template <class T>
void rk3_step(const Config& c, Field<T>& Un, double dt) {
  Field<T> L(c, 5), U1(c, 5), U2(c, 5);
  const auto interior = [&](auto&& body) {
    for (int m = 0; m < 5; ++m)
      for (int k = 0; k < c.n[2]; ++k)
        for (int j = 0; j < c.n[1]; ++j)
          for (int i = 0; i < c.n[0]; ++i) body(m, i, j, k);
  };
  fill_ghosts(Un, c);
  rhs(c, Un, L);
  interior([&](int m, int i, int j, int k) { U1(m, i, j, k) = Un(m, i, j, k) + dt * L(m, i, j, k); });
  fill_ghosts(U1, c);
  rhs(c, U1, L);
  interior([&](int m, int i, int j, int k) {
    U2(m, i, j, k) = 0.75 * Un(m, i, j, k) + 0.25 * (U1(m, i, j, k) + dt * L(m, i, j, k));
  });
  fill_ghosts(U2, c);
  rhs(c, U2, L);
  interior([&](int m, int i, int j, int k) {
    Un(m, i, j, k) = (1.0 / 3.0) * Un(m, i, j, k) + (2.0 / 3.0) * (U2(m, i, j, k) + dt * L(m, i, j, k));
  });
  fill_ghosts(Un, c);
}

// Table 2 time integrators other than TVD-RK3, with fixed dt:
//   TVD-RK2 (Gottlieb & Shu 1998), Shu-Osher form:
//     U1 = Un + dt L(Un);  U^{n+1} = 1/2 Un + 1/2 (U1 + dt L(U1))
//   Euler:  U^{n+1} = Un + dt L(Un)
template <class T>
void rk2_step(const Config& c, Field<T>& Un, double dt) {
  Field<T> L(c, 5), U1(c, 5);
  fill_ghosts(Un, c);
  rhs(c, Un, L);
  for (int m = 0; m < 5; ++m)
    for (int k = 0; k < c.n[2]; ++k)
      for (int j = 0; j < c.n[1]; ++j)
        for (int i = 0; i < c.n[0]; ++i) U1(m, i, j, k) = Un(m, i, j, k) + dt * L(m, i, j, k);
  fill_ghosts(U1, c);
  rhs(c, U1, L);
  for (int m = 0; m < 5; ++m)
    for (int k = 0; k < c.n[2]; ++k)
      for (int j = 0; j < c.n[1]; ++j)
        for (int i = 0; i < c.n[0]; ++i)
          Un(m, i, j, k) = 0.5 * Un(m, i, j, k) + 0.5 * (U1(m, i, j, k) + dt * L(m, i, j, k));
  fill_ghosts(Un, c);
}
template <class T>
void euler_step(const Config& c, Field<T>& Un, double dt) {
  Field<T> L(c, 5);
  fill_ghosts(Un, c);
  rhs(c, Un, L);
  for (int m = 0; m < 5; ++m)
    for (int k = 0; k < c.n[2]; ++k)
      for (int j = 0; j < c.n[1]; ++j)
        for (int i = 0; i < c.n[0]; ++i) Un(m, i, j, k) = Un(m, i, j, k) + dt * L(m, i, j, k);
  fill_ghosts(Un, c);
}
// One step of the configuration's integrator.
template <class T>
void time_step(const Config& c, Field<T>& Un, double dt) {
  if (c.integrator == TIME_RK2) rk2_step(c, Un, dt);
  else if (c.integrator == TIME_EULER) euler_step(c, Un, dt);
  else rk3_step(c, Un, dt);
}

// Time step (Section 3.2 names a CFL criterion and defers its formula).
// Reading used throughout this project:
//   dt_c = min_d dx_d / max_cells max_d (|u_d| + c)      (active axes d)
//   dt_v = 3/14 min_d dx_d^2 / max_cells max(mu / rho, lambda / (rho c_v)),
//          c_v = R / (gamma - 1)                         (dissipative runs only)
//   dt   = CFL min(dt_c, dt_v)
// All in FP64 from the state at the start of the step.
struct Rates { double conv, diff; };
inline Rates max_rates(const Config& c, const Field<double>& U) {
  Rates r{0.0, 0.0};
  const double lambda = conductivity(c);
  const double mu = c.viscous ? c.mu : 0.0;
  const double cv = c.R / (c.gamma - 1.0);
  for (int k = 0; k < c.n[2]; ++k)
    for (int j = 0; j < c.n[1]; ++j)
      for (int i = 0; i < c.n[0]; ++i) {
        const double rho = U(0, i, j, k);
        const double vel[3] = {U(1, i, j, k) / rho, U(2, i, j, k) / rho, U(3, i, j, k) / rho};
        const double p = (c.gamma - 1.0) *
                         (U(4, i, j, k) - 0.5 * rho * (vel[0] * vel[0] + vel[1] * vel[1] + vel[2] * vel[2]));
        const double cs = std::sqrt(c.gamma * p / rho);
        for (int d = 0; d < 3; ++d)
          if (active(c, d)) r.conv = std::max(r.conv, std::fabs(vel[d]) + cs);
        r.diff = std::max(r.diff, std::max(mu / rho, lambda / (rho * cv)));
      }
  return r;
}
inline double compute_dt(const Config& c, const Field<double>& U) {
  const Rates r = max_rates(c, U);
  double hmin = 1e300;
  for (int d = 0; d < 3; ++d)
    if (active(c, d)) hmin = std::min(hmin, spacing(c, d));
  double dt = hmin / r.conv;
  if (r.diff > 0.0) dt = std::min(dt, (3.0 / 14.0) * hmin * hmin / r.diff);
  return c.cfl * dt;
}

}  // namespace orc

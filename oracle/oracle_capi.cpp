// C entry points of the oracle, loaded with ctypes by oracle/__init__.py.
//
// TEST INFRASTRUCTURE ONLY (see jf_oracle.hpp).  Arrays are interior-only
// structure-of-arrays U[5][nz][ny][nx] in FP64, x fastest.
#include <cstring>
#include <type_traits>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

#include "dual.hpp"
#include "exact_riemann.hpp"
#include "jf_oracle.hpp"

namespace orc {

// Operation-counting scalar: every +, -, *, / and sqrt on a Counted value is
// one floating-point operation.  Used to state the algorithmic operation count
// of the scheme as defined (one evaluation per face, Eq. (FVD)).
struct Counted {
  double v;
  static long long& ops() { static long long n = 0; return n; }
  Counted() : v(0.0) {}
  Counted(double x) : v(x) {}  // NOLINT
};
#define ORC_BIN(op)                                                                     \
  inline Counted operator op(const Counted& a, const Counted& b) { ++Counted::ops(); return Counted(a.v op b.v); } \
  inline Counted operator op(const Counted& a, double b) { ++Counted::ops(); return Counted(a.v op b); }           \
  inline Counted operator op(double a, const Counted& b) { ++Counted::ops(); return Counted(a op b.v); }
ORC_BIN(+)
ORC_BIN(-)
ORC_BIN(*)
ORC_BIN(/)
#undef ORC_BIN
inline Counted operator-(const Counted& a) { return Counted(-a.v); }
inline Counted& operator+=(Counted& a, const Counted& b) { a = a + b; return a; }
inline Counted& operator-=(Counted& a, const Counted& b) { a = a - b; return a; }
inline bool operator<(const Counted& a, const Counted& b) { return a.v < b.v; }
inline bool operator>(const Counted& a, double b) { return a.v > b; }
inline bool operator>=(const Counted& a, double b) { return a.v >= b; }
inline Counted sqrt(const Counted& a) { ++Counted::ops(); return Counted(std::sqrt(a.v)); }
inline bool operator<=(const Counted& a, const Counted& b) { return a.v <= b.v; }
inline bool operator<=(const Counted& a, double b) { return a.v <= b; }
inline Counted fabs(const Counted& a) { return Counted(std::fabs(a.v)); }  // sign only: not counted
inline Counted exp(const Counted& a) { ++Counted::ops(); return Counted(std::exp(a.v)); }
inline Counted log(const Counted& a) { ++Counted::ops(); return Counted(std::log(a.v)); }

template <class T>
static void store_state(const Config& c, const Field<T>& f, double* U, double* V) {
  const size_t N = (size_t)c.n[0] * c.n[1] * c.n[2];
  for (int m = 0; m < 5; ++m)
    for (int k = 0; k < c.n[2]; ++k)
      for (int j = 0; j < c.n[1]; ++j)
        for (int i = 0; i < c.n[0]; ++i) {
          const size_t q = m * N + ((size_t)k * c.n[1] + j) * c.n[0] + i;
          const T& x = f(m, i, j, k);
          if constexpr (std::is_same<T, Dual>::value) {
            U[q] = x.v;
            if (V) V[q] = x.d;
          } else {
            U[q] = x;
          }
        }
}

static bool valid(const Config* c) {
  if (!c) return false;
  for (int d = 0; d < 3; ++d) {
    if (c->n[d] < 1) return false;
    if (c->n[d] > 1 && c->n[d] < NG) return false;  // WENO5 needs 3 distinct cells
    if (!(c->hi[d] > c->lo[d])) return false;
    const bool p0 = c->bc[2 * d] == BC_PERIODIC, p1 = c->bc[2 * d + 1] == BC_PERIODIC;
    if (p0 != p1) return false;  // periodic must be set on both sides
  }
  if (c->flux < FLUX_HLLC || c->flux > FLUX_RUSANOV_NN) return false;
  if (c->flux == FLUX_RUSANOV_NN && !c->nn) return false;
  if (c->recon < RECON_WENO5_JS || c->recon > RECON_WENO3_JS) return false;
  for (int k = 0; k < 6; ++k)
    if (c->bc[k] < BC_PERIODIC || c->bc[k] > BC_WALL) return false;
  if (c->speeds < SPEED_EINFELDT || c->speeds > SPEED_TORO) return false;
  if (c->integrator < TIME_RK3 || c->integrator > TIME_EULER) return false;
  return true;
}

}  // namespace orc

using namespace orc;

extern "C" {

// Number of OpenMP threads the oracle's loops use (1 = serial); returns the
// number in effect.
int orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

// dU/dt = L(U), Eq. (FVD).
int orc_rhs(const Config* c, const double* U, double* dUdt) {
  if (!valid(c)) return -1;
  Field<double> f(*c, 5), r(*c, 5);
  load_state(*c, U, f);
  rhs(*c, f, r);
  store_state(*c, r, dUdt, nullptr);
  return 0;
}

// Time step from the CFL criterion (reading in jf_oracle.hpp).
double orc_compute_dt(const Config* c, const double* U) {
  if (!valid(c)) return -1.0;
  Field<double> f(*c, 5);
  load_state(*c, U, f);
  return compute_dt(*c, f);
}

// nsteps TVD-RK3 steps in place.  dt > 0: fixed step; dt <= 0: CFL step each
// step, clipped so that the run ends exactly at t_end when t_end > 0 (then
// nsteps is an upper bound).  Returns the number of steps taken and writes the
// final time.
int orc_run(const Config* c, double* U, int nsteps, double dt, double t_end, double* t_out) {
  if (!valid(c)) return -1;
  Field<double> f(*c, 5);
  load_state(*c, U, f);
  double t = 0.0;
  int s = 0;
  for (; s < nsteps; ++s) {
    if (t_end > 0.0 && t >= t_end) break;
    double h = dt > 0.0 ? dt : compute_dt(*c, f);
    if (t_end > 0.0 && t + h > t_end) h = t_end - t;
    time_step(*c, f, h);
    t += h;
  }
  store_state(*c, f, U, nullptr);
  if (t_out) *t_out = t;
  return s;
}

// Forward-mode derivative of nsteps fixed-dt steps: on return U holds the
// state after the steps and V holds J V0, J the Jacobian of the steps at U0.
int orc_jvp_run(const Config* c, double* U, double* V, int nsteps, double dt) {
  if (!valid(c) || !(dt > 0.0)) return -1;
  const size_t N = (size_t)c->n[0] * c->n[1] * c->n[2];
  std::vector<Dual> ud(5 * N);
  for (size_t q = 0; q < 5 * N; ++q) ud[q] = Dual(U[q], V[q]);
  Field<Dual> f(*c, 5);
  load_state(*c, ud.data(), f);
  for (int s = 0; s < nsteps; ++s) time_step(*c, f, dt);
  store_state(*c, f, U, V);
  return 0;
}

// Forward-mode derivative with respect to the Rusanov-NN parameters: nsteps
// fixed-dt steps from U (tangent zero) with the parameters carrying the
// tangent theta_dot; on return U holds the state and V its derivative along
// theta_dot.
int orc_jvp_params_run(const Config* c, double* U, double* V, int nsteps, double dt, const double* theta_dot) {
  if (!valid(c) || !(dt > 0.0) || c->flux != FLUX_RUSANOV_NN || !theta_dot) return -1;
  Config cc = *c;
  cc.nn_dot = theta_dot;
  const size_t N = (size_t)c->n[0] * c->n[1] * c->n[2];
  std::vector<Dual> ud(5 * N);
  for (size_t q = 0; q < 5 * N; ++q) ud[q] = Dual(U[q], 0.0);
  Field<Dual> f(cc, 5);
  load_state(cc, ud.data(), f);
  for (int s = 0; s < nsteps; ++s) time_step(cc, f, dt);
  store_state(cc, f, U, V);
  return 0;
}

// Rusanov-NN dissipation alpha for given network inputs x[4].
double orc_nn_alpha(const double* theta, const double* x) { return nn_alpha(theta, x); }

// Single WENO3-JS reconstruction v^-_{i+1/2} from v[i-1..i+1].
double orc_weno3(const double* v, double eps) { return weno3_js(v[0], v[1], v[2], eps); }

// Sampled cells of a full-size run, computed one by one: for each sample
// cell, a cube of half-width 9 * nsteps + 3 cells around it is copied from U
// through the domain's boundary map (periodic wrap or zero-gradient clamp),
// nsteps fixed-dt RK3 steps are taken on that patch (the patch's own edges
// influence at most 3 cells per stage, 9 per step, so the centre cell is exact)
// and the centre cell's 5 values are written to out[5 * s + m].  idx holds
// (i, j, k) per sample.  With nsteps == 0 the right-hand side L(U) at the
// sample cell is written instead (patch half-width 3).
int orc_sample_cells(const Config* c, const double* U, int nsamples, const int* idx, int nsteps, double dt,
                     double* out) {
  if (!valid(c) || nsamples < 0 || nsteps < 0) return -1;
  const size_t N = (size_t)c->n[0] * c->n[1] * c->n[2];
  const int radius = nsteps == 0 ? 3 : 9 * nsteps + 3;
  int fail = 0;
#pragma omp parallel for schedule(dynamic)
  for (int s = 0; s < nsamples; ++s) {
    Config pc = *c;
    int lo[3];
    for (int d = 0; d < 3; ++d) {
      if (c->n[d] > 1) {
        pc.n[d] = 2 * radius + 1;
        lo[d] = idx[3 * s + d] - radius;
        const double h = spacing(*c, d);
        pc.lo[d] = 0.0;
        pc.hi[d] = h * pc.n[d];
        pc.bc[2 * d] = pc.bc[2 * d + 1] = BC_ZERO_GRADIENT;
      } else {
        lo[d] = 0;
      }
    }
    const size_t M = (size_t)pc.n[0] * pc.n[1] * pc.n[2];
    std::vector<double> patch(5 * M);
    for (int k = 0; k < pc.n[2]; ++k)
      for (int j = 0; j < pc.n[1]; ++j)
        for (int i = 0; i < pc.n[0]; ++i) {
          int g[3] = {lo[0] + i, lo[1] + j, lo[2] + k};
          for (int d = 0; d < 3; ++d) {
            const int n = c->n[d];
            if (c->bc[2 * d] == BC_PERIODIC) g[d] = ((g[d] % n) + n) % n;
            else g[d] = g[d] < 0 ? 0 : (g[d] >= n ? n - 1 : g[d]);
          }
          const size_t src = ((size_t)g[2] * c->n[1] + g[1]) * c->n[0] + g[0];
          const size_t dst = ((size_t)k * pc.n[1] + j) * pc.n[0] + i;
          for (int m = 0; m < 5; ++m) patch[m * M + dst] = U[m * N + src];
        }
    Field<double> f(pc, 5);
    load_state(pc, patch.data(), f);
    const int ci = c->n[0] > 1 ? radius : 0, cj = c->n[1] > 1 ? radius : 0, ck = c->n[2] > 1 ? radius : 0;
    if (nsteps == 0) {
      Field<double> r(pc, 5);
      rhs(pc, f, r);
      for (int m = 0; m < 5; ++m) out[5 * s + m] = r(m, ci, cj, ck);
    } else {
      for (int q = 0; q < nsteps; ++q) time_step(pc, f, dt);
      for (int m = 0; m < 5; ++m) out[5 * s + m] = f(m, ci, cj, ck);
    }
    if (!(pc.n[0] > 0)) fail = 1;
  }
  return fail ? -1 : 0;
}

// Single WENO5-JS reconstruction v^-_{i+1/2} from v[i-2..i+2].
double orc_weno5(const double* v, double eps) { return weno5_js(v[0], v[1], v[2], v[3], v[4], eps); }

// Single HLLC flux along axis d from primitive states W = [rho, u, v, w, p].
void orc_hllc(const double* WL, const double* WR, int d, double gamma, double* F) {
  hllc_flux(WL, WR, d, gamma, F);
}

// Single WENO5-Z reconstruction v^-_{i+1/2} from v[i-2..i+2].
double orc_weno5_z(const double* v, double eps) { return weno5_z(v[0], v[1], v[2], v[3], v[4], eps); }

// Signal speed estimate `kind` (SPEED_*): out = (S_L, S_R).
void orc_signal_speeds(const double* WL, const double* WR, int d, double gamma, int kind, double* out) {
  double UL[5], UR[5];
  conservative_of(WL, gamma, UL);
  conservative_of(WR, gamma, UR);
  signal_speeds(WL, WR, UL[4], UR[4], d, gamma, kind, out[0], out[1]);
}

// Toro's shock/rarefaction factor q_K for a given star pressure.
double orc_toro_q(double p_star, double pK, double gamma) { return toro_q(p_star, pK, gamma); }

// Riemann flux of kind `flux` (FLUX_*) with signal speeds `speeds` (SPEED_*).
void orc_flux(const double* WL, const double* WR, int d, double gamma, int flux, int speeds, double* F) {
  Config c{};
  c.gamma = gamma;
  c.flux = flux;
  c.speeds = speeds;
  riemann_flux(c, WL, WR, d, F);
}

// Roe eigensystem at a face along d: lambda[5], R[25] and L[25] row-major.
void orc_roe_eigensystem(const double* WL, const double* WR, int d, double gamma, double* lambda, double* R,
                         double* L) {
  const Eigensystem<double> es = roe_eigensystem(WL, WR, d, gamma);
  for (int i = 0; i < 5; ++i) {
    lambda[i] = es.lambda[i];
    for (int j = 0; j < 5; ++j) {
      R[5 * i + j] = es.R[i][j];
      L[5 * i + j] = es.L[i][j];
    }
  }
}

// Flux-splitting (ROE setup) face flux of a 1D stencil of six primitive
// states W6[6][5] (cells i-2 .. i+3 of the face x_{i+1/2}) along d.
void orc_fs_flux(const double* W6, int d, double gamma, double eps, int recon, double* F) {
  Config c{};
  c.n[0] = 6;
  c.n[1] = c.n[2] = 1;
  c.hi[0] = c.hi[1] = c.hi[2] = 1.0;
  for (int k = 0; k < 6; ++k) c.bc[k] = BC_ZERO_GRADIENT;
  c.gamma = gamma;
  c.eps = eps;
  c.recon = recon;
  c.flux = FLUX_ROE_FS;
  // the stencil along x (d = 0 layout), velocities permuted so that the
  // normal component of axis d sits in the x slot
  Field<double> W(c, 5);
  for (int j = 0; j < 6; ++j)
    for (int m = 0; m < 5; ++m) W(m, j, 0, 0) = W6[5 * j + m];
  if (d != 0) {
    for (int j = 0; j < 6; ++j) {
      const double un = W6[5 * j + 1 + d], ut1 = W6[5 * j + 1 + (d + 1) % 3], ut2 = W6[5 * j + 1 + (d + 2) % 3];
      W(1, j, 0, 0) = un;
      W(2, j, 0, 0) = ut1;
      W(3, j, 0, 0) = ut2;
    }
  }
  double G[5];
  flux_splitting_face_flux(W, c, 0, Cell(2, 0, 0), G);
  F[0] = G[0];
  F[4] = G[4];
  F[1 + d] = G[1];
  F[1 + (d + 1) % 3] = G[2];
  F[1 + (d + 2) % 3] = G[3];
}

// Single Rusanov-NN flux along axis d with network parameters theta.
void orc_flux_nn(const double* WL, const double* WR, int d, double gamma, const double* theta, double* F) {
  Config c{};
  c.gamma = gamma;
  c.flux = FLUX_RUSANOV_NN;
  c.nn = theta;
  riemann_flux(c, WL, WR, d, F);
}

// HLL flux for given signal speeds (S_L, S_R).
void orc_hll_speeds(const double* WL, const double* WR, int d, double gamma, double SL, double SR, double* F) {
  hll_flux_speeds(WL, WR, d, gamma, SL, SR, F);
}

// Exact Riemann problem: star state (p*, u*, rho*_L, rho*_R).  Returns 0, or -1
// on vacuum / failure.
int orc_exact_star(const double* WL, const double* WR, double gamma, double* out) {
  ExactRiemann er{Prim1{WL[0], WL[1], WL[2]}, Prim1{WR[0], WR[1], WR[2]}, gamma};
  if (!er.solve()) return -1;
  out[0] = er.pstar;
  out[1] = er.ustar;
  out[2] = er.star_density(er.L);
  out[3] = er.star_density(er.R);
  return 0;
}

// Exact solution (rho, u, p) at points x[0..n) and time t > 0, diaphragm at x0.
int orc_exact_sample(const double* WL, const double* WR, double gamma, double x0, double t, int n,
                     const double* x, double* W) {
  ExactRiemann er{Prim1{WL[0], WL[1], WL[2]}, Prim1{WR[0], WR[1], WR[2]}, gamma};
  if (!er.solve() || !(t > 0.0)) return -1;
  for (int q = 0; q < n; ++q) {
    const Prim1 s = er.sample((x[q] - x0) / t);
    W[3 * q + 0] = s.rho;
    W[3 * q + 1] = s.u;
    W[3 * q + 2] = s.p;
  }
  return 0;
}

// Floating-point operations of the scheme as defined, per interior cell and
// per RHS evaluation, for the configuration's active axes and physics:
// out[0] primitives (per cell), out[1] convective flux (per face, summed over
// the active axes), out[2] dissipative flux (per face, summed over the active
// axes), out[3] net flux and divergence (per cell), out[4] total per cell per
// RHS (one face per cell and axis), out[5] RK3 stage combination averaged over
// the three stages (per cell).
int orc_count_flops(const Config* c, double* out) {
  if (!valid(c)) return -1;
  Config s = *c;
  for (int d = 0; d < 3; ++d) s.n[d] = c->n[d] > 1 ? 8 : 1;
  Field<Counted> U(s, 5), W(s, 6);
  // smooth positive state so every branch is a typical one
  for (int k = 0; k < s.n[2]; ++k)
    for (int j = 0; j < s.n[1]; ++j)
      for (int i = 0; i < s.n[0]; ++i) {
        const double x = 0.3 * i + 0.2 * j + 0.1 * k;
        const double rho = 1.0 + 0.1 * std::sin(x), u = 0.1 * std::cos(x), v = 0.05 * std::sin(2 * x),
                     w = 0.02 * std::cos(3 * x), p = 1.0 + 0.1 * std::cos(x);
        U(0, i, j, k) = rho;
        U(1, i, j, k) = rho * u;
        U(2, i, j, k) = rho * v;
        U(3, i, j, k) = rho * w;
        U(4, i, j, k) = p / (s.gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w);
      }
  fill_ghosts(U, s);
  long long& ops = Counted::ops();
  ops = 0;
  primitives(U, W, s);
  const long long ncells_padded = (long long)U.s[0] * U.s[1] * U.s[2];
  const double prim = (double)ops / (double)ncells_padded;
  double conv = 0.0, diss = 0.0;
  int nact = 0;
  const bool dissipative = (s.viscous || s.heat) && s.mu != 0.0;
  for (int d = 0; d < 3; ++d) {
    if (!active(s, d)) continue;
    ++nact;
    Counted F[5], Fd[5];
    const Cell cell(3, s.n[1] > 1 ? 3 : 0, s.n[2] > 1 ? 3 : 0);
    if (s.convective) {
      ops = 0;
      convective_face_flux(W, s, d, cell, F);
      conv += (double)ops;
    }
    if (dissipative) {
      ops = 0;
      dissipative_face_flux(W, s, d, cell, Fd);
      diss += (double)ops;
    }
  }
  const double netdiv = nact * (5.0 /*F^d - F*/ + 5.0 * 2.0 /*difference and 1/dx*/ + 5.0 /*accumulate*/);
  out[0] = prim;
  out[1] = conv;
  out[2] = diss;
  out[3] = netdiv;
  out[4] = prim + conv + diss + netdiv;
  // stage 1: 2 ops, stages 2 and 3: 5 ops, per component
  out[5] = 5.0 * (2.0 + 5.0 + 5.0) / 3.0;
  return 0;
}

}  // extern "C"

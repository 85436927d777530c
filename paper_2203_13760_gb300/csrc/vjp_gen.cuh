// Adjoint (vector-Jacobian product) of one Shu-Osher stage for the run-time
// schemes the tiled adjoint of vjp.cuh does not cover: slip walls, WENO3-JS
// and the Rusanov-NN flux of Section 7.4 (with its parameter gradient), for
// inviscid 1D, 2D and 3D grids.
//
// One stage computes, as the tiled adjoint does (with one more addend),
//   out = a1 x1 + a2 x2 + a3 x3 + m + dt J(Us)^T m,   m = s_in lam,
// with J the Jacobian of the right-hand side L of Eq. (FVD) at Us.
//
// Layout of the work.  A point-wise launch writes the addends and m; then one
// thread per face (every face of every active direction) recomputes the
// face's stencil (6 cells along the normal, mapped through the boundary
// condition), its reconstruction and flux, and runs the reverse pass:
// face cotangent Fb = dt (m_right - m_left) / h (a ghost cell has no
// right-hand side, so its m is 0), flux -> reconstructed states -> stencil
// primitives -> stencil conservative states, each added to `out` of the cell
// the stencil cell maps to (global atomics; with a wall the mirrored normal
// momentum carries its sign back).  For the Rusanov-NN flux the thread also
// writes the face's network input x and the cotangent of the dissipation,
// abar = -1/2 Fb . (U_R - U_L), so that a second launch can form the
// parameter gradient sum_f abar_f d alpha(x_f) / d theta.
//
// This path is built for the small grids of the learned-flux experiment: a
// face thread redoes the full stencil work and the atomics serialise on
// shared cells, which the tiled adjoint avoids.  Atomic summation makes the
// last bits vary from run to run.
#pragma once
#include "stage.cuh"
#include "vjp_math.cuh"

namespace jf {

template <typename T>
struct GVjpArgs {
  const T* Us;        // stage state, [5][nz][ny][nx]
  const T* lam;       // cotangent of the stage output
  const T* x1;        // point-wise addends (may be null)
  const T* x2;
  const T* x3;
  T* out;
  const double* dt;
  T s_in, a1, a2, a3;
  int n[3];
  long long N;
  int periodic[3];
  int wall[3];        // bit 0: wall at the low side, bit 1: at the high side
  T inv_h[3];
  long long nface[3]; // faces per direction (0 for inactive directions)
  T* rec;             // Rusanov-NN: 5 values per face (x0..x3, abar), else null
};

// Up to kMax grids per launch (a batch, or one grid), passed by value in the
// kernel parameters: the grids' arguments and the prefix sums of their faces
// and cells, so that one launch covers every face (cell) of every grid.
template <typename T>
struct GVjpBatch {
  static constexpr int kMax = 32;
  int nsim;
  long long face_base[kMax + 1];
  long long cell_base[kMax + 1];
  GVjpArgs<T> sim[kMax];
};

// The grid an index of [0, base[nsim]) belongs to (base ascending).
__device__ __forceinline__ int find_sim(const long long* base, int nsim, long long i) {
  int lo = 0, hi = nsim - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (base[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// out = a1 x1 + a2 x2 + a3 x3 + s_in lam, every cell of every grid
template <typename T>
__global__ void __launch_bounds__(256) gvjp_point_kernel(const GVjpBatch<T> B) {
  const long long total = B.cell_base[B.nsim];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int s = find_sim(B.cell_base, B.nsim, i);
    const GVjpArgs<T>& A = B.sim[s];
    const long long c = i - B.cell_base[s];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const long long q = c + k * A.N;
      T o = A.s_in * A.lam[q];
      if (A.x1) o += A.a1 * A.x1[q];
      if (A.x2) o += A.a2 * A.x2[q];
      if (A.x3) o += A.a3 * A.x3[q];
      A.out[q] = o;
    }
  }
}

// Cotangent of W = (rho, u, v, w, p) -> cotangent of U = (rho, rho u, rho v,
// rho w, E) for an ideal gas, p = (gamma - 1) (E - |m|^2 / (2 rho)).
template <typename T>
JF_HD void prim_vjp(const T U[5], const Gas<T>& g, const T Wb[5], T Ub[5]) {
  const T ir = T(1) / U[0];
  const T u = U[1] * ir, v = U[2] * ir, w = U[3] * ir;
  const T k = g.gm1;
  Ub[0] = Wb[0] - (Wb[1] * u + Wb[2] * v + Wb[3] * w) * ir + Wb[4] * k * T(0.5) * (u * u + v * v + w * w);
  Ub[1] = Wb[1] * ir - Wb[4] * k * u;
  Ub[2] = Wb[2] * ir - Wb[4] * k * v;
  Ub[3] = Wb[3] * ir - Wb[4] * k * w;
  Ub[4] = Wb[4] * k;
}

// Reverse of side_flux<T, D> (flux F and conservative state U of one face
// side from its primitive state W): Wb += (dF/dW)^T Fb + (dU/dW)^T Ub.
template <typename T, int D>
JF_HD void side_flux_vjp(const T W[5], const Gas<T>& g, const T Fb[5], const T Ub[5], T Wb[5]) {
  const T r = W[0], un = W[1 + D], p = W[4];
  const T q2 = W[1] * W[1] + W[2] * W[2] + W[3] * W[3];
  const T E = p * g.inv_gm1 + T(0.5) * r * q2;
  const T mass = r * un;
  const T massb = Fb[0] + Fb[1] * W[1] + Fb[2] * W[2] + Fb[3] * W[3];
  T ub[3] = {Fb[1] * mass + Ub[1] * r, Fb[2] * mass + Ub[2] * r, Fb[3] * mass + Ub[3] * r};
  T pb = Fb[1 + D] + Fb[4] * un;
  T unb = Fb[4] * (E + p) + massb * r;
  const T Eb = Fb[4] * un + Ub[4];
  T rb = Ub[0] + Ub[1] * W[1] + Ub[2] * W[2] + Ub[3] * W[3] + massb * un + Eb * T(0.5) * q2;
  ub[D] += unb;
#pragma unroll
  for (int k = 0; k < 3; ++k) ub[k] += Eb * r * W[1 + k];
  pb += Eb * g.inv_gm1;
  Wb[0] += rb;
  Wb[1] += ub[0];
  Wb[2] += ub[1];
  Wb[3] += ub[2];
  Wb[4] += pb;
}

// row[0 .. NN_HIDDEN) -> registers
template <typename T>
__device__ __forceinline__ void ld_row(const T* row, T v[NN_HIDDEN]) {
#pragma unroll
  for (int j = 0; j < NN_HIDDEN; j += 4) ld4(row + j, v + j);
}
// sum_j w[j] v[j] with the weight row w read four at a time
template <typename T>
__device__ __forceinline__ T dot_row(const T* w, const T v[NN_HIDDEN], T acc) {
#pragma unroll
  for (int j = 0; j < NN_HIDDEN; j += 4) {
    T q[4];
    ld4(w + j, q);
    acc += q[0] * v[j] + q[1] * v[j + 1] + q[2] * v[j + 2] + q[3] * v[j + 3];
  }
  return acc;
}
// acc[j] += s w[j] over a weight row w
template <typename T>
__device__ __forceinline__ void axpy_row(const T* w, T s, T acc[NN_HIDDEN]) {
#pragma unroll
  for (int j = 0; j < NN_HIDDEN; j += 4) {
    T q[4];
    ld4(w + j, q);
#pragma unroll
    for (int m = 0; m < 4; ++m) acc[j + m] += s * q[m];
  }
}

// Row pitch of the per-thread hidden rows (a multiple of 4 for the vector
// loads; 36 puts the 16-byte accesses of 8 consecutive threads on distinct
// banks).
constexpr int kHRow = NN_HIDDEN + 4;

// alpha = exp(NN(x)) (as nn_alpha) and dx = d alpha / dx.  th: the
// parameters in shared memory; h1, h2: this thread's two hidden rows (kHRow
// pitch, shared memory).  Each layer's input is held in registers while its
// outputs are formed one weight row at a time; the reverse passes run over
// weight rows too (output cotangent times row added into register
// accumulators), so every parameter is read as part of a 16-byte row load.
template <typename T>
__device__ __forceinline__ T nn_alpha_grad(const T* th, const T x[4], T dx[4], T* h1, T* h2) {
  const T* W1 = th;
  const T* b1 = W1 + NN_HIDDEN * 4;
  const T* W2 = b1 + NN_HIDDEN;
  const T* b2 = W2 + NN_HIDDEN * NN_HIDDEN;
  const T* W3 = b2 + NN_HIDDEN;
  const T* b3 = W3 + NN_HIDDEN * NN_HIDDEN;
  const T* W4 = b3 + NN_HIDDEN;
  const T b4 = W4[NN_HIDDEN];
  unsigned m1 = 0, m2 = 0, m3 = 0;  // ReLU masks (bit i: unit i active)
  // layer 1 -> h1
#pragma unroll 4
  for (int i = 0; i < NN_HIDDEN; ++i) {
    T w[4];
    ld4(W1 + 4 * i, w);
    const T z = b1[i] + w[0] * x[0] + w[1] * x[1] + w[2] * x[2] + w[3] * x[3];
    h1[i] = tmax(T(0), z);
    m1 |= (z > T(0) ? 1u : 0u) << i;
  }
  T v[NN_HIDDEN];
  // layer 2 -> h2
  ld_row(h1, v);
#pragma unroll 2
  for (int i = 0; i < NN_HIDDEN; ++i) {
    const T z = dot_row(W2 + NN_HIDDEN * i, v, b2[i]);
    h2[i] = tmax(T(0), z);
    m2 |= (z > T(0) ? 1u : 0u) << i;
  }
  // layer 3 and the output
  ld_row(h2, v);
  T o = b4;
#pragma unroll 2
  for (int i = 0; i < NN_HIDDEN; ++i) {
    const T z = dot_row(W3 + NN_HIDDEN * i, v, b3[i]);
    o += W4[i] * tmax(T(0), z);
    m3 |= (z > T(0) ? 1u : 0u) << i;
  }
  const T alpha = texp(o);
  // reverse, seed d alpha / d o = alpha: cotangent of layer 2's outputs
  // (v, then masked into h2) = sum over active layer-3 units i of
  // alpha W4[i] W3[i][:]
#pragma unroll
  for (int j = 0; j < NN_HIDDEN; ++j) v[j] = T(0);
#pragma unroll 2
  for (int i = 0; i < NN_HIDDEN; ++i)
    if ((m3 >> i) & 1u) axpy_row(W3 + NN_HIDDEN * i, alpha * W4[i], v);
#pragma unroll
  for (int j = 0; j < NN_HIDDEN; ++j) h2[j] = (m2 >> j) & 1u ? v[j] : T(0);
  // cotangent of layer 1's outputs = sum_j h2[j] W2[j][:], masked
#pragma unroll
  for (int k = 0; k < NN_HIDDEN; ++k) v[k] = T(0);
#pragma unroll 2
  for (int j = 0; j < NN_HIDDEN; ++j) {
    const T s = h2[j];
    if (s != T(0)) axpy_row(W2 + NN_HIDDEN * j, s, v);
  }
  dx[0] = dx[1] = dx[2] = dx[3] = T(0);
#pragma unroll
  for (int k = 0; k < NN_HIDDEN; ++k) {
    const T s = (m1 >> k) & 1u ? v[k] : T(0);
    T w[4];
    ld4(W1 + 4 * k, w);
#pragma unroll
    for (int m = 0; m < 4; ++m) dx[m] += w[m] * s;
  }
  return alpha;
}

// Reverse of rusanov_nn<T, D>: WLb, WRb += cotangents; rec = (x, abar).
template <typename T, int D>
__device__ __forceinline__ void rusanov_nn_vjp(const T WL[5], const T WR[5], const Gas<T>& g, const T* th,
                                               const T Fb[5], T WLb[5], T WRb[5], T rec[5], T* h1, T* h2) {
  T EL, ER, irL, irR, cL, cR;
  side_state(WL, g, EL, irL, cL);
  side_state(WR, g, ER, irR, cR);
  T x[4], dx[4];
  nn_inputs<T, D>(WL, WR, g, cL, cR, x);
  const T alpha = nn_alpha_grad(th, x, dx, h1, h2);
  T FL[5], FR[5], UL[5], UR[5];
  side_flux<T, D>(WL, EL, FL, UL);
  side_flux<T, D>(WR, ER, FR, UR);
  T abar = T(0), hFb[5], ULb[5], URb[5];
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    abar -= T(0.5) * Fb[q] * (UR[q] - UL[q]);
    hFb[q] = T(0.5) * Fb[q];
    ULb[q] = T(0.5) * alpha * Fb[q];
    URb[q] = -ULb[q];
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) rec[m] = x[m];
  rec[4] = abar;
  side_flux_vjp<T, D>(WL, g, hFb, ULb, WLb);
  side_flux_vjp<T, D>(WR, g, hFb, URb, WRb);
  // through alpha(x): xb = abar d alpha / dx
  T xb[4];
#pragma unroll
  for (int m = 0; m < 4; ++m) xb[m] = abar * dx[m];
  const T du = WR[1 + D] - WL[1 + D];
  const T s0 = du < T(0) ? T(-1) : T(1);  // d|y|/dy, taken as +1 at 0
  WLb[1 + D] += -s0 * xb[0] + T(0.5) * xb[1];
  WRb[1 + D] += s0 * xb[0] + T(0.5) * xb[1];
  // mean sound speed, c = sqrt(gamma p / rho): dc/dp = c / (2 p), dc/drho = -c / (2 rho)
  const T cb = T(0.5) * xb[2];
  WLb[4] += cb * cL / (T(2) * WL[4]);
  WLb[0] -= cb * cL / (T(2) * WL[0]);
  WRb[4] += cb * cR / (T(2) * WR[4]);
  WRb[0] -= cb * cR / (T(2) * WR[0]);
  // entropy jump, s = (ln p - gamma ln rho) / (gamma - 1)
  const T sL = (tlog(WL[4]) - g.gamma * tlog(WL[0])) * g.inv_gm1;
  const T sR = (tlog(WR[4]) - g.gamma * tlog(WR[0])) * g.inv_gm1;
  const T s3 = sR - sL < T(0) ? T(-1) : T(1);
  const T sbR = s3 * xb[3], sbL = -sbR;
  WLb[4] += sbL * g.inv_gm1 / WL[4];
  WLb[0] -= sbL * g.gamma * g.inv_gm1 / WL[0];
  WRb[4] += sbR * g.inv_gm1 / WR[4];
  WRb[0] -= sbR * g.gamma * g.inv_gm1 / WR[0];
}

// WENO3-JS reverse (left-biased value from vm1, v0, vp1): vb[k] += yb dy/dv_k.
template <typename T>
JF_HD void weno3_vjp(T vm1, T v0, T vp1, T eps, T yb, T vb[3]) {
  const T q0 = T(0.5) * (T(3) * v0 - vm1), q1 = T(0.5) * (v0 + vp1);
  const T e0 = v0 - vm1, e1 = vp1 - v0;
  const T t0 = eps + e0 * e0, t1 = eps + e1 * e1;
  const T r0 = T(1) / t0, r1 = T(1) / t1;
  const T a0 = T(1.0 / 3.0) * r0 * r0, a1 = T(2.0 / 3.0) * r1 * r1;
  const T inv = T(1) / (a0 + a1);
  const T y = (a0 * q0 + a1 * q1) * inv;
  const T s = yb * inv;
  const T qb0 = s * a0, qb1 = s * a1;
  // d alpha_k / d t_k = -2 alpha_k / t_k, d t_k / d e_k = 2 e_k
  const T eb0 = -T(4) * s * (q0 - y) * a0 * r0 * e0;
  const T eb1 = -T(4) * s * (q1 - y) * a1 * r1 * e1;
  vb[0] += -T(0.5) * qb0 - eb0;
  vb[1] += T(1.5) * qb0 + T(0.5) * qb1 + eb0 - eb1;
  vb[2] += T(0.5) * qb1 + eb1;
}

// The reverse pass of one face normal to D whose right cell is c (the left
// cell is c - e_D).  RECON: 0 WENO5-JS, 2 WENO3-JS; FLUX: 0 HLLC (Einfeldt
// speeds), 4 Rusanov-NN.
template <typename T, int DIM, int RECON, int FLUX, int D>
__device__ __forceinline__ void gvjp_face(const GVjpArgs<T>& A, const Gas<T>& g, const int c[3], long long f,
                                          T* h1, T* h2) {
  const int n = A.n[D];
  const long long sD = D == 0 ? 1 : (D == 1 ? (long long)A.n[0] : (long long)A.n[0] * A.n[1]);
  long long base = 0;  // offset of the face's line (coordinate D = 0)
  {
    long long s = 1;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (a != D) base += (long long)c[a] * s;
      s *= A.n[a];
    }
  }
  // m of the two cells beside the face (a ghost has none)
  const T scale = T(*A.dt) * A.inv_h[D];
  T Fb[5];
  {
    int iL = c[D] - 1, iR = c[D];
    bool hasL = true, hasR = true;
    if (A.periodic[D]) {
      if (iL < 0) iL += n;
    } else {
      hasL = iL >= 0;
      hasR = iR < n;
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      const T mL = hasL ? A.lam[base + iL * sD + q * A.N] : T(0);
      const T mR = hasR ? A.lam[base + iR * sD + q * A.N] : T(0);
      Fb[q] = scale * A.s_in * (mR - mL);
    }
  }
  // stencil cells c[D] - 3 .. c[D] + 2 along D, through the boundary map
  // (loaded twice: for the face states, and again for the reverse pass, so
  // that the flux's reverse pass runs with few values live)
  auto stencil = [&](int j, T Uj[5], T Wj[5], long long& at, bool& fl) {
    fl = false;
    const int i = map_index_bc(c[D] - 3 + j, n, A.periodic[D], A.wall[D], fl);
    at = base + i * sD;
#pragma unroll
    for (int q = 0; q < 5; ++q) Uj[q] = A.Us[at + q * A.N];
    if (fl) Uj[1 + D] = -Uj[1 + D];
    const T ir = T(1) / Uj[0];
    Wj[0] = Uj[0];
    Wj[1] = Uj[1] * ir;
    Wj[2] = Uj[2] * ir;
    Wj[3] = Uj[3] * ir;
    Wj[4] = g.gm1 * (Uj[4] - T(0.5) * Uj[0] * (Wj[1] * Wj[1] + Wj[2] * Wj[2] + Wj[3] * Wj[3]));
  };
  // face states (stencil slot 2 is the left cell, slot 3 the right one)
  T WL[5], WR[5];
  bool fbL = false, fbR = false;  // safe-reconstruction fallback to the cell values
  {
    T W[6][5];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
      T Uj[5];
      long long at;
      bool fl;
      stencil(j, Uj, W[j], at, fl);
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      if (RECON == 2) {
        WL[q] = weno3(W[1][q], W[2][q], W[3][q], g.eps);
        WR[q] = weno3(W[4][q], W[3][q], W[2][q], g.eps);
      } else {
        WL[q] = weno5(W[0][q], W[1][q], W[2][q], W[3][q], W[4][q], g.eps, 0);
        WR[q] = weno5(W[5][q], W[4][q], W[3][q], W[2][q], W[1][q], g.eps, 0);
      }
    }
    if (g.safe) {
      fbL = !(WL[0] > T(0)) || !(WL[4] > T(0));
      fbR = !(WR[0] > T(0)) || !(WR[4] > T(0));
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        if (fbL) WL[q] = W[2][q];
        if (fbR) WR[q] = W[3][q];
      }
    }
  }
  T WLb[5] = {T(0), T(0), T(0), T(0), T(0)}, WRb[5] = {T(0), T(0), T(0), T(0), T(0)};
  if constexpr (FLUX == 4) {
    T rec[5];
    rusanov_nn_vjp<T, D>(WL, WR, g, g.nn, Fb, WLb, WRb, rec, h1, h2);
    if (A.rec)
#pragma unroll
      for (int m = 0; m < 5; ++m) A.rec[f * 5 + m] = rec[m];
  } else {
    hllc_vjp<T, D>(WL, WR, g, Fb, WLb, WRb);
  }
  // reconstruction reverse
  T W[6][5], U[6][5], Wb[6][5];
  long long at[6];
  bool flip[6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    stencil(j, U[j], W[j], at[j], flip[j]);
#pragma unroll
    for (int q = 0; q < 5; ++q) Wb[j][q] = T(0);
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    if (fbL) {
      Wb[2][q] += WLb[q];
    } else if (RECON == 2) {
      T vb[3] = {T(0), T(0), T(0)};
      weno3_vjp(W[1][q], W[2][q], W[3][q], g.eps, WLb[q], vb);
      Wb[1][q] += vb[0]; Wb[2][q] += vb[1]; Wb[3][q] += vb[2];
    } else {
      T vb[5] = {T(0), T(0), T(0), T(0), T(0)};
      weno5_vjp(W[0][q], W[1][q], W[2][q], W[3][q], W[4][q], g.eps, WLb[q], vb);
#pragma unroll
      for (int k = 0; k < 5; ++k) Wb[k][q] += vb[k];
    }
    if (fbR) {
      Wb[3][q] += WRb[q];
    } else if (RECON == 2) {
      T vb[3] = {T(0), T(0), T(0)};
      weno3_vjp(W[4][q], W[3][q], W[2][q], g.eps, WRb[q], vb);
      Wb[4][q] += vb[0]; Wb[3][q] += vb[1]; Wb[2][q] += vb[2];
    } else {
      T vb[5] = {T(0), T(0), T(0), T(0), T(0)};
      weno5_vjp(W[5][q], W[4][q], W[3][q], W[2][q], W[1][q], g.eps, WRb[q], vb);
#pragma unroll
      for (int k = 0; k < 5; ++k) Wb[5 - k][q] += vb[k];
    }
  }
  // primitive -> conservative reverse, back through the boundary map
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    if (RECON == 2 && (j == 0 || j == 5)) continue;
    T Ub[5];
    prim_vjp(U[j], g, Wb[j], Ub);
    if (flip[j]) Ub[1 + D] = -Ub[1 + D];
#pragma unroll
    for (int q = 0; q < 5; ++q) atomicAdd(A.out + at[j] + q * A.N, Ub[q]);
  }
}

// One thread per face of every grid of the launch: within a grid, faces of
// direction 0 first, then 1, then 2; within a direction x fastest.  A periodic axis has n faces (face 0 is also face n),
// any other n + 1.  Rusanov-NN: dynamic shared memory of
// gvjp_face_smem_bytes holds the network parameters (padded to a multiple
// of 4) and each thread's two hidden-layer rows.
constexpr int kGvjpThreads = 128;
constexpr int kNnParamsPad = (NN_PARAMS + 3) / 4 * 4;
template <typename T, int FLUX>
constexpr size_t gvjp_face_smem_bytes() {
  return FLUX == 4 ? sizeof(T) * ((size_t)kNnParamsPad + (size_t)kGvjpThreads * 2 * kHRow) : 0;
}

template <typename T, int DIM, int RECON, int FLUX>
__global__ void __launch_bounds__(kGvjpThreads) gvjp_face_kernel(const GVjpBatch<T> B, const Gas<T> g) {
  extern __shared__ __align__(16) unsigned char gvjp_smem[];
  T* th = reinterpret_cast<T*>(gvjp_smem);  // the network parameters (Rusanov-NN)
  T* h1 = th + kNnParamsPad + threadIdx.x * kHRow;
  T* h2 = h1 + kGvjpThreads * kHRow;
  Gas<T> gs = g;
  if constexpr (FLUX == 4) {
    for (int i = threadIdx.x; i < NN_PARAMS; i += blockDim.x) th[i] = g.nn[i];
    __syncthreads();
    gs.nn = th;
  }
  const long long gf = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gf >= B.face_base[B.nsim]) return;
  const int sidx = find_sim(B.face_base, B.nsim, gf);
  const GVjpArgs<T>& A = B.sim[sidx];
  const long long f = gf - B.face_base[sidx];  // face of this grid (its record index)
  long long r = f;
  int d = 0;
  for (; d < DIM; ++d) {
    if (r < A.nface[d]) break;
    r -= A.nface[d];
  }
  if (d >= DIM) return;
  int ext[3] = {A.n[0], A.n[1], A.n[2]};
  ext[d] += A.periodic[d] ? 0 : 1;
  int c[3];
  c[0] = (int)(r % ext[0]);
  r /= ext[0];
  c[1] = (int)(r % ext[1]);
  c[2] = (int)(r / ext[1]);
  if (d == 0) gvjp_face<T, DIM, RECON, FLUX, 0>(A, gs, c, f, h1, h2);
  if constexpr (DIM >= 2) if (d == 1) gvjp_face<T, DIM, RECON, FLUX, 1>(A, gs, c, f, h1, h2);
  if constexpr (DIM == 3) if (d == 2) gvjp_face<T, DIM, RECON, FLUX, 2>(A, gs, c, f, h1, h2);
}

// Parameter gradient of the Rusanov-NN dissipation: grad += sum over the
// face records (x_f, abar_f) of abar_f d alpha(x_f) / d theta.
//
// Persistent blocks of kNnWarps warps; the block stages theta in shared
// memory, and each warp takes chunks of 32 records (one per lane).  Per
// chunk, each lane evaluates the network of its record and the cotangents of
// every layer (seed d alpha / d o = alpha, scaled by abar) into shared rows of
// 33 (conflict-free), reusing rows once they are consumed; then lane L adds
// row L of every weight gradient summed over the 32 records
// (dW[L][k] = sum_f G[f][L] H[f][k]) to accumulators kept in registers across
// chunks.  At the end the block sums its warps' accumulators in shared memory
// and adds them to grad with one atomic per parameter.
constexpr int kNnRow = NN_HIDDEN + 1;
constexpr int kNnWarps = 4;
constexpr int kNnWarpElems = 4 * 32 * kNnRow + 32 * 5;  // four row sets, inputs, output cotangents
template <typename T>
constexpr size_t nn_grad_smem_bytes() {
  return sizeof(T) * (size_t)(NN_PARAMS + kNnWarps * kNnWarpElems);
}

template <typename T>
__global__ void __launch_bounds__(32 * kNnWarps) nn_param_grad_kernel(const T* __restrict__ theta,
                                                                      const T* __restrict__ rec, long long nrec,
                                                                      T* grad) {
  extern __shared__ __align__(16) unsigned char nn_smem[];
  T* TH = reinterpret_cast<T*>(nn_smem);
  for (int i = threadIdx.x; i < NN_PARAMS; i += blockDim.x) TH[i] = theta[i];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* base = TH + NN_PARAMS + warp * kNnWarpElems;
  T* R1 = base;                 // H1
  T* R2 = R1 + 32 * kNnRow;     // H2
  T* R3 = R2 + 32 * kNnRow;     // H3, then G2
  T* R4 = R3 + 32 * kNnRow;     // G3, then G1
  T* X = R4 + 32 * kNnRow;      // [32][4]
  T* OB = X + 32 * 4;           // [32]
  const T* W1 = TH;
  const T* b1 = W1 + NN_HIDDEN * 4;
  const T* W2 = b1 + NN_HIDDEN;
  const T* b2 = W2 + NN_HIDDEN * NN_HIDDEN;
  const T* W3 = b2 + NN_HIDDEN;
  const T* b3 = W3 + NN_HIDDEN * NN_HIDDEN;
  const T* W4 = b3 + NN_HIDDEN;
  __syncthreads();
  // row `lane` of every gradient, accumulated over this warp's chunks
  T a3[NN_HIDDEN], a2[NN_HIDDEN], a1[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
  for (int k = 0; k < NN_HIDDEN; ++k) a3[k] = a2[k] = T(0);
  T ab1 = T(0), ab2 = T(0), ab3 = T(0), a4 = T(0), ab4 = T(0);
  const long long nchunk = (nrec + 31) / 32;
  T* h1 = R1 + lane * kNnRow;
  T* h2 = R2 + lane * kNnRow;
  T* r3 = R3 + lane * kNnRow;
  T* r4 = R4 + lane * kNnRow;
  for (long long ch = (long long)blockIdx.x * kNnWarps + warp; ch < nchunk; ch += (long long)gridDim.x * kNnWarps) {
    const long long f = ch * 32 + lane;
    T x[4] = {T(0), T(0), T(0), T(0)}, abar = T(0);
    if (f < nrec) {
#pragma unroll
      for (int m = 0; m < 4; ++m) x[m] = rec[f * 5 + m];
      abar = rec[f * 5 + 4];
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) X[lane * 4 + m] = x[m];
    // forward: h1, h2, h3 (r3); each layer's input in registers (v), the
    // weight rows read four at a time from the shared copy of theta
    T v[NN_HIDDEN];
#pragma unroll 4
    for (int i = 0; i < NN_HIDDEN; ++i) {
      T w[4];
      ld4(W1 + 4 * i, w);
      h1[i] = tmax(T(0), b1[i] + w[0] * x[0] + w[1] * x[1] + w[2] * x[2] + w[3] * x[3]);
    }
#pragma unroll
    for (int j = 0; j < NN_HIDDEN; ++j) v[j] = h1[j];
#pragma unroll 2
    for (int i = 0; i < NN_HIDDEN; ++i) h2[i] = tmax(T(0), dot_row(W2 + NN_HIDDEN * i, v, b2[i]));
#pragma unroll
    for (int j = 0; j < NN_HIDDEN; ++j) v[j] = h2[j];
    T o = W4[NN_HIDDEN];
#pragma unroll 2
    for (int i = 0; i < NN_HIDDEN; ++i) {
      const T h3 = tmax(T(0), dot_row(W3 + NN_HIDDEN * i, v, b3[i]));
      r3[i] = h3;
      o += W4[i] * h3;
    }
    const T ob = f < nrec ? abar * texp(o) : T(0);  // d alpha / d o = alpha
    OB[lane] = ob;
#pragma unroll 4
    for (int i = 0; i < NN_HIDDEN; ++i) r4[i] = r3[i] > T(0) ? ob * W4[i] : T(0);  // G3
    __syncwarp();
    // layers 4 and 3 (H3 in R3, G3 in R4, H2 in R2)
#pragma unroll 1
    for (int r = 0; r < 32; ++r) {
      const T g3 = R4[r * kNnRow + lane];
      ab3 += g3;
      a4 += OB[r] * R3[r * kNnRow + lane];
      if (lane == 0) ab4 += OB[r];
#pragma unroll
      for (int k = 0; k < NN_HIDDEN; ++k) a3[k] += g3 * R2[r * kNnRow + k];
    }
    __syncwarp();
    // G2 into R3: g2[j] = [h2_j > 0] sum_i W3[i][j] g3[i] (row updates of v)
#pragma unroll
    for (int j = 0; j < NN_HIDDEN; ++j) v[j] = T(0);
#pragma unroll 2
    for (int i = 0; i < NN_HIDDEN; ++i) axpy_row(W3 + NN_HIDDEN * i, r4[i], v);
#pragma unroll
    for (int j = 0; j < NN_HIDDEN; ++j) r3[j] = h2[j] > T(0) ? v[j] : T(0);
    __syncwarp();
    // layer 2 (G2 in R3, H1 in R1)
#pragma unroll 1
    for (int r = 0; r < 32; ++r) {
      const T g2 = R3[r * kNnRow + lane];
      ab2 += g2;
#pragma unroll
      for (int k = 0; k < NN_HIDDEN; ++k) a2[k] += g2 * R1[r * kNnRow + k];
    }
    __syncwarp();
    // G1 into R4: g1[k] = [h1_k > 0] sum_j W2[j][k] g2[j] (row updates of v)
#pragma unroll
    for (int k = 0; k < NN_HIDDEN; ++k) v[k] = T(0);
#pragma unroll 2
    for (int j = 0; j < NN_HIDDEN; ++j) axpy_row(W2 + NN_HIDDEN * j, r3[j], v);
#pragma unroll
    for (int k = 0; k < NN_HIDDEN; ++k) r4[k] = h1[k] > T(0) ? v[k] : T(0);
    __syncwarp();
    // layer 1 (G1 in R4, inputs in X)
#pragma unroll 1
    for (int r = 0; r < 32; ++r) {
      const T g1 = R4[r * kNnRow + lane];
      ab1 += g1;
#pragma unroll
      for (int m = 0; m < 4; ++m) a1[m] += g1 * X[r * 4 + m];
    }
    __syncwarp();
  }
  // block sum of the warps' rows (the row sets are free now), then one
  // atomic per parameter
  __syncthreads();
  T* S = TH + NN_PARAMS;  // [kNnWarps][NN_PARAMS]
  T* Sw = S + warp * NN_PARAMS;
  const int L = lane;
#pragma unroll
  for (int m = 0; m < 4; ++m) Sw[4 * L + m] = a1[m];
  Sw[NN_HIDDEN * 4 + L] = ab1;
  T* sW2 = Sw + NN_HIDDEN * 4 + NN_HIDDEN;
#pragma unroll
  for (int k = 0; k < NN_HIDDEN; ++k) sW2[NN_HIDDEN * L + k] = a2[k];
  sW2[NN_HIDDEN * NN_HIDDEN + L] = ab2;
  T* sW3 = sW2 + NN_HIDDEN * NN_HIDDEN + NN_HIDDEN;
#pragma unroll
  for (int k = 0; k < NN_HIDDEN; ++k) sW3[NN_HIDDEN * L + k] = a3[k];
  sW3[NN_HIDDEN * NN_HIDDEN + L] = ab3;
  T* sW4 = sW3 + NN_HIDDEN * NN_HIDDEN + NN_HIDDEN;
  sW4[L] = a4;
  if (L == 0) sW4[NN_HIDDEN] = ab4;
  __syncthreads();
  for (int i = threadIdx.x; i < NN_PARAMS; i += blockDim.x) {
    T sum = T(0);
#pragma unroll
    for (int w = 0; w < kNnWarps; ++w) sum += S[w * NN_PARAMS + i];
    if (sum != T(0)) atomicAdd(grad + i, sum);
  }
}

}  // namespace jf

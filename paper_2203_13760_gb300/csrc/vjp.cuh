// Adjoint (vector-Jacobian product) of one Shu-Osher stage (Sections 3.1-3.4,
// Section 7.2).
//
// One launch computes, for every interior cell,
//   out = a1 x1 + a2 x2 + m + dt J(Us)^T m,   m = s_in lam,
// where J is the Jacobian of the right-hand side L of Eq. (FVD) at the stage
// state Us.  The adjoint of one fixed-dt RK3 step is three such launches
// (see jf_rk3_step_vjp in vjp.cu).
//
// Derivation.  L_c = sum_d (NF_d(c+1/2) - NF_d(c-1/2)) / h_d with the net face
// flux NF = F^d - F, so the face cotangent is nu_f = (m_left - m_right) / h_d
// and (J^T m)_j = (dW/dU)_j^T sum_f (dNF_f/dW_j)^T nu_f.  Each face's reverse
// pass (HLLC -> WENO5 for the convective part, the C4 stencils for the
// dissipative part) yields cotangents of the primitive variables (and T) of
// its stencil cells; the cell then applies the transposed Jacobian of
// W(U) (and of T = p / (rho R)).
//
// Tiling.  A CTA owns a BX x BY tile of cells.  It stages the primitives of a
// 5-cell halo around the tile (WENO5 of a face 3 cells outside the tile reads
// 2 more) and m with a 3-cell halo, evaluates the reverse pass of every face
// whose stencil touches a tile cell, and accumulates the resulting cotangents
// of tile cells in shared memory (shared-memory atomics: the summation order,
// and so the last bits, may vary from run to run).  Ghost cells follow the
// boundary condition: with zero gradient a ghost has no right-hand side
// (m = 0) and its cotangent goes to the interior cell it copies; with periodic
// wrap every ghost face is a real face that the owning tile also evaluates,
// so only cotangents of the tile's own cells are kept.
#pragma once
#include "stage.cuh"
#include "vjp_math.cuh"

namespace jf {

template <typename T>
struct VjpArgs {
  const T* Us;        // stage state, [5][nz][ny][nx]
  const T* lam;       // cotangent of the stage output
  const T* x1;        // point-wise addends (may be null)
  const T* x2;
  T* out;
  const double* dt;
  T s_in, a1, a2;
  int nx, ny;
  long long N;
  int periodic[2];
  T inv_h[2];
  int* flag;
};

template <int BX, int BY, int DIM, bool VISC>
struct VGeo {
  static constexpr int H = 5;                         // W halo
  static constexpr int HY = DIM >= 2 ? H : 0;
  static constexpr int PX = BX + 2 * H, PY = BY + 2 * HY, CS = PX * PY;
  static constexpr int NCW = VISC ? 6 : 5;
  static constexpr int MH = 3;                        // m halo
  static constexpr int MHY = DIM >= 2 ? MH : 0;
  static constexpr int MPX = BX + 2 * MH, MPY = BY + 2 * MHY, MCS = MPX * MPY;
  static constexpr int NCELL = BX * BY;
  static constexpr int NT = BX * BY;
  static constexpr int VR = DIM >= 2 ? 2 : 0;         // viscous faces reach 2 rows beyond the tile
};

template <typename T, int DIM, bool VISC, int BX, int BY>
constexpr size_t vjp_smem_bytes() {
  using G = VGeo<BX, BY, DIM, VISC>;
  return sizeof(T) * (size_t)(G::NCW * G::CS + 5 * G::MCS + 6 * G::NCELL);
}

// Shared-memory views and the boundary-aware accumulator of one tile.
template <typename T, int DIM, bool VISC, int BX, int BY>
struct VTile {
  using G = VGeo<BX, BY, DIM, VISC>;
  const T* W;   // [NCW][PY][PX], tile cell (0, 0) at (H, HY)
  const T* M;   // [5][MPY][MPX], tile cell (0, 0) at (MH, MHY)
  T* acc;       // [6][BY][BX]
  int gx0, gy0, nx, ny, px, py;

  __device__ __forceinline__ T w(int c, int x, int y) const { return W[c * G::CS + (y + G::HY) * G::PX + x + G::H]; }
  __device__ __forceinline__ T m(int c, int x, int y) const {
    return M[c * G::MCS + (y + G::MHY) * G::MPX + x + G::MH];
  }
  // target tile column of tile-relative column x, or -1 if the cotangent is
  // not this tile's to keep
  __device__ __forceinline__ int owner(int x, int x0, int n, int periodic, int B) const {
    const int gxx = x0 + x;
    if (periodic) return (x >= 0 && x < B && gxx < n) ? x : -1;
    const int c = gxx < 0 ? 0 : (gxx >= n ? n - 1 : gxx);
    const int t = c - x0;
    return (t >= 0 && t < B) ? t : -1;
  }
  __device__ __forceinline__ void add(int c, int x, int y, T v) const {
    const int tx = owner(x, gx0, nx, px, BX);
    const int ty = DIM >= 2 ? owner(y, gy0, ny, py, BY) : 0;
    if (tx >= 0 && ty >= 0) atomicAdd(acc + (c * BY + ty) * BX + tx, v);
  }
};

// In-plane axis roles for a face normal to axis d (runtime): offsets (along
// the normal, along the tangent) -> tile (x, y).
__device__ __forceinline__ void vroles(int d, int n, int t, int& x, int& y) {
  x = d == 0 ? n : t;
  y = d == 0 ? t : n;
}

// Reverse pass of the convective flux of the face between tile cells
// (x0, y0) and its neighbour along axis d; nu = dLoss/dNF (NF = -F + ...).
// HLLC is evaluated in the face frame (normal velocity first), which is the
// same function of the rotated state, so one instance serves both axes.
template <typename T, int DIM, bool VISC, int BX, int BY>
__device__ __forceinline__ void conv_face_vjp(const VTile<T, DIM, VISC, BX, BY>& V, int d, int x0, int y0,
                                           const T nu[5], const Gas<T>& g) {
  auto at = [&](int c, int n) -> T {
    int x, y;
    vroles(d, n, 0, x, y);
    return V.w(c, x0 + x, y0 + y);
  };
  const int cn = 1 + d, ct = 2 - d;  // normal / tangential velocity components (2D)
  T Wm[5], Wp[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    const int pc = c == 1 ? cn : (c == 2 ? ct : c);  // face-frame order
    Wm[c] = weno5(at(pc, -2), at(pc, -1), at(pc, 0), at(pc, 1), at(pc, 2), g.eps);
    Wp[c] = weno5(at(pc, 3), at(pc, 2), at(pc, 1), at(pc, 0), at(pc, -1), g.eps);
  }
  bool fm = false, fp = false;
  if (g.safe) {
    fm = !(Wm[0] > T(0)) || !(Wm[4] > T(0));
    fp = !(Wp[0] > T(0)) || !(Wp[4] > T(0));
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const int pc = c == 1 ? cn : (c == 2 ? ct : c);
      if (fm) Wm[c] = at(pc, 0);
      if (fp) Wp[c] = at(pc, 1);
    }
  }
  T Fb[5], Wmb[5], Wpb[5];
  Fb[0] = -nu[0];
  Fb[1] = -(d == 0 ? nu[1] : nu[2]);
  Fb[2] = -(d == 0 ? nu[2] : nu[1]);
  Fb[3] = -nu[3];
  Fb[4] = -nu[4];
  hllc_vjp<T, 0>(Wm, Wp, g, Fb, Wmb, Wpb);
#pragma unroll 1
  for (int c = 0; c < 5; ++c) {
    const int pc = c == 1 ? cn : (c == 2 ? ct : c);
    const T bm = c == 0 ? Wmb[0] : c == 1 ? Wmb[1] : c == 2 ? Wmb[2] : c == 3 ? Wmb[3] : Wmb[4];
    const T bp = c == 0 ? Wpb[0] : c == 1 ? Wpb[1] : c == 2 ? Wpb[2] : c == 3 ? Wpb[3] : Wpb[4];
    T v[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) v[q] = at(pc, q - 2);
    T vb[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    if (fm) {
      vb[2] += bm;
    } else {
      T t[5] = {T(0), T(0), T(0), T(0), T(0)};
      weno5_vjp(v[0], v[1], v[2], v[3], v[4], g.eps, bm, t);
#pragma unroll
      for (int q = 0; q < 5; ++q) vb[q] += t[q];
    }
    if (fp) {
      vb[3] += bp;
    } else {
      T t[5] = {T(0), T(0), T(0), T(0), T(0)};
      weno5_vjp(v[5], v[4], v[3], v[2], v[1], g.eps, bp, t);
#pragma unroll
      for (int q = 0; q < 5; ++q) vb[5 - q] += t[q];
    }
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      int x, y;
      vroles(d, q - 2, 0, x, y);
      V.add(pc, x0 + x, y0 + y, vb[q]);
    }
  }
}

// Reverse pass of the dissipative flux of the same face (NF = ... + F^d),
// in the face frame: n = normal axis d, t = the other in-plane axis, z = the
// out-of-plane axis (no derivatives along it in 2D).  Forward (Sections 2,
// 3.4): du_k/dn = DF4(u_k), dT/dn = DF4(T); du_n/dt and du_t/dt by DC4 at
// the cells -1..2 along n, interpolated with RC4; face velocities RC4(u_k);
// tau_n = mu (2 du_n/dn - 2/3 div), tau_t = mu (du_n/dt + du_t/dn),
// tau_z = mu du_z/dn, div = du_n/dn + du_t/dt;
// F^d = [0, tau, u_f . tau + lambda dT/dn] (tau_n in component 1 + d).
template <typename T, int DIM, bool VISC, int BX, int BY>
__device__ __forceinline__ void visc_face_vjp(const VTile<T, DIM, VISC, BX, BY>& V, int d, int x0, int y0,
                                           const T nu[5], const Gas<T>& g, const T inv_h[2]) {
  auto at = [&](int c, int n, int t) -> T {
    int x, y;
    vroles(d, n, t, x, y);
    return V.w(c, x0 + x, y0 + y);
  };
  auto put = [&](int c, int n, int t, T val) {
    int x, y;
    vroles(d, n, t, x, y);
    V.add(c, x0 + x, y0 + y, val);
  };
  const int cn = 1 + d, ct = 2 - d, cz = 3;
  const T hn = d == 0 ? inv_h[0] : inv_h[1];
  const T ht = d == 0 ? inv_h[1] : inv_h[0];
  const T df[4] = {T(1) / T(24), -T(27) / T(24), T(27) / T(24), -T(1) / T(24)};
  const T rc[4] = {-T(1) / T(16), T(9) / T(16), T(9) / T(16), -T(1) / T(16)};
  const T dcw[4] = {T(1) / T(12), -T(8) / T(12), T(8) / T(12), -T(1) / T(12)};
  const int dco[4] = {-2, -1, 1, 2};
  // ---- forward ----
  T gn[3], uf[3];  // d u_k / dn and face velocities, k = n, t, z
  const int comp[3] = {cn, ct, cz};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    T s = T(0), f = T(0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T u = at(comp[k], q - 1, 0);
      s += df[q] * u;
      f += rc[q] * u;
    }
    gn[k] = s * hn;
    uf[k] = f;
  }
  T gnt = T(0), gtt = T(0);  // d u_n / dt, d u_t / dt
  if (DIM >= 2) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      T acc = T(0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        T cen = T(0);
#pragma unroll
        for (int j = 0; j < 4; ++j) cen += dcw[j] * at(comp[k], q - 1, dco[j]);
        acc += rc[q] * cen;
      }
      if (k == 0) gnt = acc * ht; else gtt = acc * ht;
    }
  }
  const T div = gn[0] + gtt;
  const T tau[3] = {g.mu * (T(2) * gn[0]) - (T(2) / T(3)) * g.mu * div, g.mu * (gnt + gn[1]), g.mu * gn[2]};
  // ---- reverse ----
  const T nun[3] = {nu[cn], nu[ct], nu[cz]};
  T taub[3], ufb[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    taub[k] = nun[k] + nu[4] * uf[k];
    ufb[k] = nu[4] * tau[k];
  }
  const T dTb = nu[4] * g.lambda;
  const T divb = -(T(2) / T(3)) * g.mu * taub[0];
  const T gnb[3] = {T(2) * g.mu * taub[0] + divb, g.mu * taub[1], g.mu * taub[2]};
  const T gntb = g.mu * taub[1], gttb = divb;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
#pragma unroll
    for (int k = 0; k < 3; ++k) put(comp[k], q - 1, 0, gnb[k] * hn * df[q] + ufb[k] * rc[q]);
    put(5, q - 1, 0, dTb * hn * df[q]);
  }
  if (DIM >= 2) {
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const T gb = (k == 0 ? gntb : gttb) * ht;
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int j = 0; j < 4; ++j) put(comp[k], q - 1, dco[j], gb * rc[q] * dcw[j]);
    }
  }
}

// The stage VJP kernel (DIM = 1 or 2).  blockDim.x == BX * BY,
// grid = (ceil(nx/BX), ceil(ny/BY)).
template <typename T, int DIM, bool VISC, int BX, int BY>
__global__ void __launch_bounds__(BX * BY, 2) vjp_stage_kernel(const VjpArgs<T> A, const Gas<T> g) {
  using G = VGeo<BX, BY, DIM, VISC>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Wb = reinterpret_cast<T*>(smem_raw);
  T* Mb = Wb + G::NCW * G::CS;
  T* acc = Mb + 5 * G::MCS;
  const int gx0 = blockIdx.x * BX, gy0 = blockIdx.y * BY;
  const int tid = threadIdx.x;

  // stage W (halo 5) and m = s_in lam (halo 3; zero on zero-gradient ghosts)
  bool bad = false;
  for (int t = tid; t < G::CS; t += G::NT) {
    const int ly = t / G::PX, lx = t - ly * G::PX;
    const int gx = map_index(gx0 + lx - G::H, A.nx, A.periodic[0]);
    const int gy = DIM >= 2 ? map_index(gy0 + ly - G::HY, A.ny, A.periodic[1]) : 0;
    const long long q = (long long)gy * A.nx + gx;
    const T r = A.Us[q];
    const T inv = T(1) / r;
    const T u = A.Us[q + A.N] * inv, v = A.Us[q + 2 * A.N] * inv, w = A.Us[q + 3 * A.N] * inv;
    const T p = g.gm1 * (A.Us[q + 4 * A.N] - T(0.5) * r * (u * u + v * v + w * w));
    bad |= !(r > T(0)) || !(p > T(0));
    Wb[t] = r;
    Wb[G::CS + t] = u;
    Wb[2 * G::CS + t] = v;
    Wb[3 * G::CS + t] = w;
    Wb[4 * G::CS + t] = p;
    if (VISC) Wb[5 * G::CS + t] = p * inv * g.inv_R;
  }
  if (bad) atomicOr(A.flag, 1);
  for (int t = tid; t < G::MCS; t += G::NT) {
    const int ly = t / G::MPX, lx = t - ly * G::MPX;
    const int rx = gx0 + lx - G::MH, ry = DIM >= 2 ? gy0 + ly - G::MHY : 0;
    const bool ghost = (!A.periodic[0] && (rx < 0 || rx >= A.nx)) ||
                       (DIM >= 2 && !A.periodic[1] && (ry < 0 || ry >= A.ny));
    const int gx = map_index(rx, A.nx, A.periodic[0]);
    const int gy = DIM >= 2 ? map_index(ry, A.ny, A.periodic[1]) : 0;
    const long long q = (long long)gy * A.nx + gx;
#pragma unroll
    for (int c = 0; c < 5; ++c) Mb[c * G::MCS + t] = ghost ? T(0) : A.s_in * A.lam[q + c * A.N];
  }
  for (int t = tid; t < 6 * G::NCELL; t += G::NT) acc[t] = T(0);
  __syncthreads();

  VTile<T, DIM, VISC, BX, BY> V{Wb, Mb, acc, gx0, gy0, A.nx, A.ny, A.periodic[0], DIM >= 2 ? A.periodic[1] : 1};
  const T inv_h[2] = {A.inv_h[0], A.inv_h[1]};

  // convective faces along x: tile rows, left cells x = -3 .. BX+1 (a face
  // reaches cells x-2 .. x+3)
  for (int f = tid; f < BY * (BX + 5); f += G::NT) {
    const int y = f / (BX + 5), x = f - y * (BX + 5) - 3;
    T nu[5];
    bool any = false;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      nu[c] = (V.m(c, x, y) - V.m(c, x + 1, y)) * inv_h[0];
      any |= nu[c] != T(0);
    }
    if (any) conv_face_vjp<T, DIM, VISC, BX, BY>(V, 0, x, y, nu, g);
  }
  if (DIM >= 2) {
    // convective faces along y: tile columns, lower cells y = -3 .. BY+1
    for (int f = tid; f < BX * (BY + 5); f += G::NT) {
      const int yy = f / BX, x = f - yy * BX, y = yy - 3;
      T nu[5];
      bool any = false;
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        nu[c] = (V.m(c, x, y) - V.m(c, x, y + 1)) * inv_h[1];
        any |= nu[c] != T(0);
      }
      if (any) conv_face_vjp<T, DIM, VISC, BX, BY>(V, 1, x, y, nu, g);
    }
  }
  if (VISC) {
    // dissipative faces along x: rows -VR .. BY-1+VR, left cells -2 .. BX (a
    // face reaches cells x-1 .. x+2 and rows y-2 .. y+2)
    constexpr int NXR = BY + 2 * G::VR, NXC = BX + 3;
    for (int f = tid; f < NXR * NXC; f += G::NT) {
      const int yy = f / NXC, x = f - yy * NXC - 2, y = yy - G::VR;
      T nu[5];
      bool any = false;
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        nu[c] = (V.m(c, x, y) - V.m(c, x + 1, y)) * inv_h[0];
        any |= nu[c] != T(0);
      }
      if (any) visc_face_vjp<T, DIM, VISC, BX, BY>(V, 0, x, y, nu, g, inv_h);
    }
    if (DIM >= 2) {
      // dissipative faces along y: columns -2 .. BX+1, lower cells -2 .. BY
      constexpr int NYC = BX + 4, NYR = BY + 3;
      for (int f = tid; f < NYC * NYR; f += G::NT) {
        const int yy = f / NYC, x = f - yy * NYC - 2, y = yy - 2;
        T nu[5];
        bool any = false;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          nu[c] = (V.m(c, x, y) - V.m(c, x, y + 1)) * inv_h[1];
          any |= nu[c] != T(0);
        }
        if (any) visc_face_vjp<T, DIM, VISC, BX, BY>(V, 1, x, y, nu, g, inv_h);
      }
    }
  }
  __syncthreads();

  // cells: cotangent of W (+T) -> cotangent of U, then the stage combination
  const int tx = tid % BX, ty = tid / BX;
  const int gx = gx0 + tx, gy = gy0 + ty;
  if (gx < A.nx && gy < (DIM >= 2 ? A.ny : 1)) {
    const T r = V.w(0, tx, ty), u = V.w(1, tx, ty), v = V.w(2, tx, ty), w = V.w(3, tx, ty), p = V.w(4, tx, ty);
    const int cell = ty * BX + tx;
    T br = acc[cell], bu = acc[G::NCELL + cell], bv = acc[2 * G::NCELL + cell], bw = acc[3 * G::NCELL + cell];
    T bp = acc[4 * G::NCELL + cell];
    if (VISC) {
      const T bT = acc[5 * G::NCELL + cell];
      const T Tc = V.w(5, tx, ty);
      br -= bT * Tc / r;       // T = p / (rho R)
      bp += bT * Tc / p;
    }
    const T inv = T(1) / r;
    T bU[5];
    bU[0] = br - (bu * u + bv * v + bw * w) * inv + bp * g.gm1 * T(0.5) * (u * u + v * v + w * w);
    bU[1] = bu * inv - bp * g.gm1 * u;
    bU[2] = bv * inv - bp * g.gm1 * v;
    bU[3] = bw * inv - bp * g.gm1 * w;
    bU[4] = bp * g.gm1;
    const T dt = T(*A.dt);
    const long long q = (long long)gy * A.nx + gx;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      T o = V.m(c, tx, ty) + dt * bU[c];
      if (A.x1) o += A.a1 * A.x1[q + c * A.N];
      if (A.x2) o += A.a2 * A.x2[q + c * A.N];
      A.out[q + c * A.N] = o;
    }
  }
}

}  // namespace jf

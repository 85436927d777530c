// Adjoint (vector-Jacobian product) of one Shu-Osher stage (Sections 3.1-3.4,
// Section 7.2): the per-face reverse passes, and the box kernel that runs
// them on 1D and 2D grids (3D grids: the z-marching kernel of vjp3.cuh,
// which calls the same reverse passes).
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
// Tiling.  A CTA owns a BX (x BY) box of cells.  It stages the primitives of
// a 5-cell halo around the box on every active axis (WENO5 of a face 3 cells
// outside reads 2 more) and m with a 3-cell halo, evaluates the reverse pass
// of every face whose stencil touches a cell of the box, and accumulates the
// resulting cotangents in shared memory (shared-memory atomics: the
// summation order, and so the last bits, may vary from run to run).
// Ghost cells follow the boundary condition: with zero gradient a ghost has
// no right-hand side (m = 0) and its cotangent goes to the interior cell it
// copies; with periodic wrap every ghost face is a real face that the owning
// box also evaluates, so only cotangents of the box's own cells are kept.
// The accumulator covers the box and a 5-cell halo, so an addition needs no
// ownership test; boxes near a non-periodic boundary fold their ghost cells
// afterwards.  In 2D the viscous tangential stencil is applied in two
// separable steps (cell-centre derivative cotangents, then a gather pass) and
// the face tasks are ordered for conflict-free banks.
//
// Faces are handled in their own frame (normal axis d, tangential axes t1,
// t2): HLLC of the rotated state (normal velocity first) and the viscous
// stress in face coordinates, so one instance of each reverse pass serves
// every axis.
#pragma once
#include "stage.cuh"
#include <type_traits>

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
  int n[3];
  long long N;
  int periodic[3];
  T inv_h[3];
  int* flag;
};

template <int BX, int BY, int BZ, int DIM, bool VISC>
struct VGeo {
  static constexpr int HX = 5, HY = DIM >= 2 ? 5 : 0, HZ = 0;  // W halo
  static constexpr int PX = BX + 2 * HX, PY = BY + 2 * HY, PZ = BZ + 2 * HZ, CS = PX * PY * PZ;
  static constexpr int NCW = VISC ? 6 : 5;
  static constexpr int MX = 3, MY = DIM >= 2 ? 3 : 0, MZ = 0;  // m halo
  static constexpr int MPX = BX + 2 * MX, MPY = BY + 2 * MY, MPZ = BZ + 2 * MZ, MCS = MPX * MPY * MPZ;
  static constexpr int NCELL = BX * BY * BZ;
  static constexpr int NT = NCELL;
  // cotangents accumulate over the box and a 5-cell halo (every cell a face's
  // stencil reaches), with no ownership test per addition; boxes near a
  // non-periodic boundary fold ghost cells onto the cells they copy afterwards
  static constexpr int AX = 5, AY = DIM >= 2 ? 5 : 0;
  static constexpr int APX = BX + 2 * AX, APY = BY + 2 * AY, ACS = APX * APY;
  // 2D viscous: the tangential C4 stencil (DC4 along the tangent at the cells
  // -1..2 along the normal, then RC4 to the face) is separable, so a face
  // adds its cotangents of the four cell-centre derivatives (slots
  // d * 2 + k: k = 0 for du_n/de, 1 for du_e/de) and one gather pass applies
  // the transposed DC4 afterwards: 8 instead of 32 additions per face.
  static constexpr int NCB = DIM == 2 && VISC ? 4 : 0;
  static_assert(DIM <= 2, "3D grids take the z-marching kernel (vjp3.cuh)");
  static_assert(DIM >= 2 || BY == 1, "1D boxes are one row");
  static_assert(BZ == 1, "boxes are one plane");
};

template <typename T, int DIM, bool VISC, int BX, int BY, int BZ>
constexpr size_t vjp_smem_bytes() {
  using G = VGeo<BX, BY, BZ, DIM, VISC>;
  return sizeof(T) * (size_t)(G::NCW * G::CS + 5 * G::MCS + (6 + G::NCB) * G::ACS);
}

// Position along the axes of a face frame: offset n along the normal d, a
// along t1, b along t2, for axis `axis` of (x, y, z).
struct Frame {
  int d, t1, t2;
  __device__ __forceinline__ int pick(int axis, int n, int a, int b) const {
    return axis == d ? n : (axis == t1 ? a : b);
  }
};

// Face-task counts of a box per direction (zero for inactive directions).
template <int DIM, int BX, int BY, int BZ>
struct VCount {
  static constexpr int B(int a) { return a == 0 ? BX : (a == 1 ? BY : BZ); }
  static constexpr int conv(int d) {
    return d < DIM ? (B(d) + 5) * ((d + 1) % 3 < DIM ? B((d + 1) % 3) : 1) * ((d + 2) % 3 < DIM ? B((d + 2) % 3) : 1)
                   : 0;
  }
  static constexpr int visc(int d) {
    return d < DIM ? (B(d) + 3) * ((d + 1) % 3 < DIM ? B((d + 1) % 3) + 4 : 1) *
                         ((d + 2) % 3 < DIM ? B((d + 2) % 3) + 4 : 1)
                   : 0;
  }
};

// 2D task order: a face family covers R rows (y) by C columns (x) of faces.
// Task f goes to row r and column c (0-based) so that a warp takes 16
// consecutive rows of two adjacent columns: every shared array of a box has a
// row pitch of 2 (mod 4) words (26 or 22), so the 16 rows of one column fall
// on 16 distinct even banks (plus the column) and the next column on the odd
// ones, and the warp's loads and atomics are free of bank conflicts.  Rows
// beyond the first 16 follow as a second block in row-fastest order.
template <int R, int C>
__device__ __forceinline__ void task_rc(int f, int& r, int& c) {
  constexpr int RA = R >= 16 ? 16 : 0;
  constexpr int RB = R - RA > 0 ? R - RA : 1;  // rows of the second block (none when R == 16)
  if (f < RA * C) {
    r = f % 16;
    c = f / 16;
  } else {
    const int g = f - RA * C;
    r = RA + g % RB;
    c = g / RB;
  }
}

// Shared-memory views and the boundary-aware accumulator of one box.
template <typename T, int DIM, bool VISC, int BX, int BY, int BZ>
struct VTile {
  using G = VGeo<BX, BY, BZ, DIM, VISC>;
  static constexpr int NCB = G::NCB;
  static constexpr bool SEP3 = false;
  __device__ __forceinline__ void add_sep(int, int, int, int, int, int, T) const {}
  const T* W;   // [NCW][PY][PX], box cell (0, 0) at (HX, HY)
  const T* M;   // [5][MPY][MPX]
  T* acc;       // [6][APY][APX], box cell (0, 0) at (AX, AY)
  T* cb;        // [NCB][APY][APX]: cotangents of cell-centre tangential derivatives (2D viscous)
  int g0[3], n[3], per[3];

  // coordinates along inactive axes are always 0: fold them at compile time
  __device__ __forceinline__ T w(int c, int x, int y, int) const {
    const int yy = DIM >= 2 ? y : 0;
    return W[c * G::CS + (yy + G::HY) * G::PX + x + G::HX];
  }
  __device__ __forceinline__ T m(int c, int x, int y, int) const {
    const int yy = DIM >= 2 ? y : 0;
    return M[c * G::MCS + (yy + G::MY) * G::MPX + x + G::MX];
  }
  // box coordinate that keeps a cotangent landing on box-relative coordinate
  // x along an axis, or -1 if it is not this box's to keep
  __device__ __forceinline__ int owner(int x, int x0, int nn, int periodic, int B) const {
    const int gxx = x0 + x;
    if (periodic) return (x >= 0 && x < B && gxx < nn) ? x : -1;
    const int c = gxx < 0 ? 0 : (gxx >= nn ? nn - 1 : gxx);
    const int t = c - x0;
    return (t >= 0 && t < B) ? t : -1;
  }
  __device__ __forceinline__ void add(int c, int x, int y, int, T v) const {
    const int yy = DIM >= 2 ? y : 0;
    atomicAdd(acc + c * G::ACS + (yy + G::AY) * G::APX + x + G::AX, v);
  }
  __device__ __forceinline__ void add_cb(int slot, int x, int y, T v) const {
    atomicAdd(cb + slot * G::ACS + (y + G::AY) * G::APX + x + G::AX, v);
  }
};

template <typename T>
__device__ __forceinline__ T sel3(const T v[5], int i) {  // v[i], i in 1..3, without dynamic indexing
  return i == 1 ? v[1] : (i == 2 ? v[2] : v[3]);
}
template <typename T>
__device__ __forceinline__ T sel5(const T v[5], int i) {
  return i == 0 ? v[0] : i == 1 ? v[1] : i == 2 ? v[2] : i == 3 ? v[3] : v[4];
}

// Reverse pass of the convective flux of the face between box cell p and its
// neighbour along F.d; nu = dLoss/dNF (NF = -F + ...).
// Tile: any accessor with w(c, x, y, z) (primitive c of a cell, tile-relative
// coordinates) and add(c, x, y, z, v) (cotangent accumulation).
template <typename T, int DIM, bool VISC, typename Tile>
__device__ __forceinline__ void conv_face_vjp(const Tile& V, const Frame& F, const int p[3], const T nu[5],
                                              const Gas<T>& g) {
  auto at = [&](int c, int s) -> T {
    return V.w(c, p[0] + F.pick(0, s, 0, 0), p[1] + F.pick(1, s, 0, 0), p[2] + F.pick(2, s, 0, 0));
  };
  const int cn = 1 + F.d, c1 = 1 + F.t1, c2 = 1 + F.t2;  // physical components of the frame velocities
  auto phys = [&](int c) { return c == 1 ? cn : (c == 2 ? c1 : (c == 3 ? c2 : c)); };
  constexpr bool PACKED = std::is_same<T, float>::value;  // FP32: both sides in FP32x2 lanes
  T Wm[5], Wp[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    const int pc = phys(c);
    if constexpr (PACKED) {
      const float2 r = weno5_pair(make_float2(at(pc, -2), at(pc, 3)), make_float2(at(pc, -1), at(pc, 2)),
                                  make_float2(at(pc, 0), at(pc, 1)), make_float2(at(pc, 1), at(pc, 0)),
                                  make_float2(at(pc, 2), at(pc, -1)), g.eps);
      Wm[c] = r.x;
      Wp[c] = r.y;
    } else {
      Wm[c] = weno5(at(pc, -2), at(pc, -1), at(pc, 0), at(pc, 1), at(pc, 2), g.eps);
      Wp[c] = weno5(at(pc, 3), at(pc, 2), at(pc, 1), at(pc, 0), at(pc, -1), g.eps);
    }
  }
  bool fm = false, fp = false;
  if (g.safe) {
    fm = !(Wm[0] > T(0)) || !(Wm[4] > T(0));
    fp = !(Wp[0] > T(0)) || !(Wp[4] > T(0));
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      if (fm) Wm[c] = at(phys(c), 0);
      if (fp) Wp[c] = at(phys(c), 1);
    }
  }
  T Fb[5], Wmb[5], Wpb[5];
  Fb[0] = -nu[0];
  Fb[1] = -sel3(nu, cn);
  Fb[2] = -sel3(nu, c1);
  Fb[3] = -sel3(nu, c2);
  Fb[4] = -nu[4];
  hllc_vjp<T, 0>(Wm, Wp, g, Fb, Wmb, Wpb);
#pragma unroll 1
  for (int c = 0; c < 5; ++c) {
    const int pc = phys(c);
    const T bm = sel5(Wmb, c), bp = sel5(Wpb, c);
    T v[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) v[q] = at(pc, q - 2);
    T vb[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
    if constexpr (PACKED) {
      float2 t2[5];
      weno5_vjp_pair(make_float2(v[0], v[5]), make_float2(v[1], v[4]), make_float2(v[2], v[3]),
                     make_float2(v[3], v[2]), make_float2(v[4], v[1]), g.eps,
                     make_float2(fm ? 0.0f : bm, fp ? 0.0f : bp), t2);
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        vb[q] += t2[q].x;
        vb[5 - q] += t2[q].y;
      }
      if (fm) vb[2] += bm;
      if (fp) vb[3] += bp;
    } else {
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
    }
#pragma unroll
    for (int q = 0; q < 6; ++q)
      V.add(pc, p[0] + F.pick(0, q - 2, 0, 0), p[1] + F.pick(1, q - 2, 0, 0), p[2] + F.pick(2, q - 2, 0, 0), vb[q]);
  }
}

// Reverse pass of the dissipative flux of the same face (NF = ... + F^d), in
// face coordinates (n = normal axis, e_j = tangential axes t1, t2, each with
// derivatives only if active).  Forward (Sections 2, 3.4):
//   du_k/dn = DF4(u_k), dT/dn = DF4(T) along the normal (k = n, t1, t2);
//   du_n/de_j and du_ej/de_j by DC4 along e_j at the cells -1..2 along n,
//   interpolated to the face with RC4; face velocities RC4(u_k);
//   div = du_n/dn + sum_j du_ej/de_j;
//   tau_n = mu (2 du_n/dn - 2/3 div), tau_ej = mu (du_n/de_j + du_ej/dn);
//   F^d = [0, tau, u_f . tau + lambda dT/dn] (tau_n in component 1 + d).
template <typename T, int DIM, bool VISC, typename Tile>
__device__ __forceinline__ void visc_face_vjp(const Tile& V, const Frame& F, const int p[3], const T nu[5],
                                              const Gas<T>& g, const T inv_h[3]) {
  auto at = [&](int c, int s, int a, int b) -> T {
    return V.w(c, p[0] + F.pick(0, s, a, b), p[1] + F.pick(1, s, a, b), p[2] + F.pick(2, s, a, b));
  };
  auto put = [&](int c, int s, int a, int b, T val) {
    V.add(c, p[0] + F.pick(0, s, a, b), p[1] + F.pick(1, s, a, b), p[2] + F.pick(2, s, a, b), val);
  };
  const int comp[3] = {1 + F.d, 1 + F.t1, 1 + F.t2};
  const bool act[2] = {F.t1 < DIM, F.t2 < DIM};
  const T hn = F.d == 0 ? inv_h[0] : (F.d == 1 ? inv_h[1] : inv_h[2]);
  const T he[2] = {F.t1 == 0 ? inv_h[0] : (F.t1 == 1 ? inv_h[1] : inv_h[2]),
                   F.t2 == 0 ? inv_h[0] : (F.t2 == 1 ? inv_h[1] : inv_h[2])};
  const T df[4] = {T(1) / T(24), -T(27) / T(24), T(27) / T(24), -T(1) / T(24)};
  const T rc[4] = {-T(1) / T(16), T(9) / T(16), T(9) / T(16), -T(1) / T(16)};
  const T dcw[4] = {T(1) / T(12), -T(8) / T(12), T(8) / T(12), -T(1) / T(12)};
  const int dco[4] = {-2, -1, 1, 2};
  // ---- forward ----
  T gn[3], uf[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    T s = T(0), f = T(0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const T u = at(comp[k], q - 1, 0, 0);
      s += df[q] * u;
      f += rc[q] * u;
    }
    gn[k] = s * hn;
    uf[k] = f;
  }
  T gt[2][2] = {{T(0), T(0)}, {T(0), T(0)}};  // [j][0] = du_n/de_j, [j][1] = du_ej/de_j
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    if (!act[j]) continue;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int c = k == 0 ? comp[0] : comp[1 + j];
      T acc = T(0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        T cen = T(0);
#pragma unroll
        for (int o = 0; o < 4; ++o)
          cen += dcw[o] * (j == 0 ? at(c, q - 1, dco[o], 0) : at(c, q - 1, 0, dco[o]));
        acc += rc[q] * cen;
      }
      gt[j][k] = acc * he[j];
    }
  }
  const T div = gn[0] + gt[0][1] + gt[1][1];
  const T tau[3] = {g.mu * (T(2) * gn[0]) - (T(2) / T(3)) * g.mu * div, g.mu * (gt[0][0] + gn[1]),
                    g.mu * (gt[1][0] + gn[2])};
  // ---- reverse ----
  const T nun[3] = {sel3(nu, comp[0]), sel3(nu, comp[1]), sel3(nu, comp[2])};
  T taub[3], ufb[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    taub[k] = nun[k] + nu[4] * uf[k];
    ufb[k] = nu[4] * tau[k];
  }
  const T dTb = nu[4] * g.lambda;
  const T divb = -(T(2) / T(3)) * g.mu * taub[0];
  const T gnb[3] = {T(2) * g.mu * taub[0] + divb, g.mu * taub[1], g.mu * taub[2]};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
#pragma unroll
    for (int k = 0; k < 3; ++k) put(comp[k], q - 1, 0, 0, gnb[k] * hn * df[q] + ufb[k] * rc[q]);
    put(5, q - 1, 0, 0, dTb * hn * df[q]);
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    if (!act[j]) continue;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int c = k == 0 ? comp[0] : comp[1 + j];
      const T gb = (k == 0 ? g.mu * taub[1 + j] : divb) * he[j];
      if constexpr (Tile::SEP3) {
        // 3D: centre-derivative cotangents by (tangent axis, component); the
        // tile spreads them along the tangent once per plane
        const int e = j == 0 ? F.t1 : F.t2;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          V.add_sep(F.d, e, c, p[0] + F.pick(0, q - 1, 0, 0), p[1] + F.pick(1, q - 1, 0, 0),
                    p[2] + F.pick(2, q - 1, 0, 0), gb * rc[q]);
      } else if constexpr (Tile::NCB > 0) {
        // centre-derivative cotangents; the gather pass spreads them along the tangent
#pragma unroll
        for (int q = 0; q < 4; ++q)
          V.add_cb(F.d * 2 + k, p[0] + F.pick(0, q - 1, 0, 0), p[1] + F.pick(1, q - 1, 0, 0), gb * rc[q]);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int o = 0; o < 4; ++o) {
            const T val = gb * rc[q] * dcw[o];
            if (j == 0) put(c, q - 1, dco[o], 0, val); else put(c, q - 1, 0, dco[o], val);
          }
      }
    }
  }
}

// The stage VJP kernel.  blockDim.x == BX * BY * BZ,
// grid = (ceil(nx/BX), ceil(ny/BY), ceil(nz/BZ)).
template <typename T, int DIM, bool VISC, int BX, int BY, int BZ, int MINB>
__global__ void __launch_bounds__(BX * BY * BZ, MINB) vjp_stage_kernel(const VjpArgs<T> A, const Gas<T> g) {
  using G = VGeo<BX, BY, BZ, DIM, VISC>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Wb = reinterpret_cast<T*>(smem_raw);
  T* Mb = Wb + G::NCW * G::CS;
  T* acc = Mb + 5 * G::MCS;
  T* cbuf = acc + 6 * G::ACS;
  const int g0[3] = {(int)blockIdx.x * BX, (int)blockIdx.y * BY, 0};
  const int tid = threadIdx.x;

  // stage W (halo 5) and m = s_in lam (halo 3; zero on zero-gradient ghosts)
  bool bad = false;
  for (int t = tid; t < G::CS; t += G::NT) {
    const int lx = t % G::PX, ly = t / G::PX;
    const int gx = map_index(g0[0] + lx - G::HX, A.n[0], A.periodic[0]);
    const int gy = DIM >= 2 ? map_index(g0[1] + ly - G::HY, A.n[1], A.periodic[1]) : 0;
    const long long q = (long long)gy * A.n[0] + gx;
    const T r = A.Us[q];
    const T inv = trcp(r);
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
    const int lx = t % G::MPX, ly = t / G::MPX;
    const int r[2] = {g0[0] + lx - G::MX, DIM >= 2 ? g0[1] + ly - G::MY : 0};
    bool ghost = false;
#pragma unroll
    for (int a = 0; a < DIM; ++a) ghost |= !A.periodic[a] && (r[a] < 0 || r[a] >= A.n[a]);
    const int gx = map_index(r[0], A.n[0], A.periodic[0]);
    const int gy = DIM >= 2 ? map_index(r[1], A.n[1], A.periodic[1]) : 0;
    const long long q = (long long)gy * A.n[0] + gx;
#pragma unroll
    for (int c = 0; c < 5; ++c) Mb[c * G::MCS + t] = ghost ? T(0) : A.s_in * A.lam[q + c * A.N];
  }
  for (int t = tid; t < (6 + G::NCB) * G::ACS; t += G::NT) acc[t] = T(0);
  __syncthreads();

  VTile<T, DIM, VISC, BX, BY, BZ> V;
  V.W = Wb;
  V.M = Mb;
  V.acc = acc;
  V.cb = cbuf;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    V.g0[a] = g0[a];
    V.n[a] = A.n[a];
    V.per[a] = a < DIM ? A.periodic[a] : 1;
  }
  const T inv_h[3] = {A.inv_h[0], A.inv_h[1], A.inv_h[2]};

  auto face_nu = [&](const Frame& F, const int p[3], T nu[5]) -> bool {
    const int q0 = p[0] + (F.d == 0), q1 = p[1] + (F.d == 1), q2 = p[2] + (F.d == 2);
    const T h = F.d == 0 ? inv_h[0] : (F.d == 1 ? inv_h[1] : inv_h[2]);
    bool any = false;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      nu[c] = (V.m(c, p[0], p[1], p[2]) - V.m(c, q0, q1, q2)) * h;
      any |= nu[c] != T(0);
    }
    return any;
  };

  // The face reverse passes of the box as one flat list of tasks, so that
  // every thread takes the same number of faces (up to one) whatever the
  // per-direction counts: convective faces of each active direction (left
  // cells -3 .. B_d+1 along d: a face reaches cells -2 .. +3 along d; the
  // box's own cells across), then, if viscous, the dissipative faces (left
  // cells -2 .. B_d along d, -2 .. B+1 across on the active tangential axes).
  // Face index -> (s along d, a along t1, b along t2): in 2D by task_rc (16
  // rows of two adjacent columns per warp); in 1D with the x
  // coordinate fastest across the lanes of a warp (x is s for d = 0, b (t2)
  // for d = 1 and a (t1) for d = 2).
  auto conv_task = [&](auto dtag, int f) {
    constexpr int d = decltype(dtag)::value;
    constexpr int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const Frame F{d, t1, t2};
    constexpr int en = VCount<DIM, BX, BY, BZ>::B(d) + 5;
    constexpr int B1 = t1 < DIM ? VCount<DIM, BX, BY, BZ>::B(t1) : 1;
    constexpr int B2 = t2 < DIM ? VCount<DIM, BX, BY, BZ>::B(t2) : 1;
    int s, a, b;
    if (DIM == 2 && d == 0) {  // rows: a (y), columns: s (x)
      int r, c;
      task_rc<B1, en>(f, r, c);
      s = c - 3;
      a = r;
      b = 0;
    } else if (DIM == 2 && d == 1) {  // rows: s (y), columns: b (x)
      int r, c;
      task_rc<en, B2>(f, r, c);
      s = r - 3;
      a = 0;
      b = c;
    } else if (d == 0) {
      s = f % en - 3;
      a = (f / en) % B1;
      b = f / (en * B1);
    } else if (d == 1) {
      b = f % B2;
      s = (f / B2) % en - 3;
      a = f / (B2 * en);
    } else {
      a = f % B1;
      b = (f / B1) % B2;
      s = f / (B1 * B2) - 3;
    }
    const int p[3] = {F.pick(0, s, a, b), F.pick(1, s, a, b), F.pick(2, s, a, b)};
    T nu[5];
    if (face_nu(F, p, nu)) conv_face_vjp<T, DIM, VISC>(V, F, p, nu, g);
  };
  auto visc_task = [&](auto dtag, int f) {
    constexpr int d = decltype(dtag)::value;
    constexpr int t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const Frame F{d, t1, t2};
    constexpr int en = VCount<DIM, BX, BY, BZ>::B(d) + 3;
    constexpr int e1 = t1 < DIM ? VCount<DIM, BX, BY, BZ>::B(t1) + 4 : 1;
    constexpr int e2 = t2 < DIM ? VCount<DIM, BX, BY, BZ>::B(t2) + 4 : 1;
    constexpr int o1 = t1 < DIM ? 2 : 0, o2 = t2 < DIM ? 2 : 0;
    int s, a, b;
    if (DIM == 2 && d == 0) {  // rows: a (y), columns: s (x)
      int r, c;
      task_rc<e1, en>(f, r, c);
      s = c - 2;
      a = r - o1;
      b = 0;
    } else if (DIM == 2 && d == 1) {  // rows: s (y), columns: b (x)
      int r, c;
      task_rc<en, e2>(f, r, c);
      s = r - 2;
      a = 0;
      b = c - o2;
    } else if (d == 0) {
      s = f % en - 2;
      a = (f / en) % e1 - o1;
      b = f / (en * e1) - o2;
    } else if (d == 1) {
      b = f % e2 - o2;
      s = (f / e2) % en - 2;
      a = f / (e2 * en) - o1;
    } else {
      a = f % e1 - o1;
      b = (f / e1) % e2 - o2;
      s = f / (e1 * e2) - 2;
    }
    const int p[3] = {F.pick(0, s, a, b), F.pick(1, s, a, b), F.pick(2, s, a, b)};
    T nu[5];
    if (face_nu(F, p, nu)) visc_face_vjp<T, DIM, VISC>(V, F, p, nu, g, inv_h);
  };
  using C = VCount<DIM, BX, BY, BZ>;
  constexpr int c0 = C::conv(0), c1 = C::conv(1), c2 = C::conv(2);
  constexpr int v0 = VISC ? C::visc(0) : 0, v1 = VISC ? C::visc(1) : 0, v2 = VISC ? C::visc(2) : 0;
  constexpr int total = c0 + c1 + c2 + v0 + v1 + v2;
  for (int f = tid; f < total; f += G::NT) {
    int r = f;
    if (r < c0) { conv_task(std::integral_constant<int, 0>{}, r); continue; }
    r -= c0;
    if constexpr (DIM >= 2) {
      if (r < c1) { conv_task(std::integral_constant<int, 1>{}, r); continue; }
      r -= c1;
    }
    if constexpr (VISC) {
      if (r < v0) { visc_task(std::integral_constant<int, 0>{}, r); continue; }
      r -= v0;
      if constexpr (DIM >= 2) {
        if (r < v1) { visc_task(std::integral_constant<int, 1>{}, r); continue; }
        r -= v1;
      }
    }
  }
  __syncthreads();

  if constexpr (G::NCB > 0) {
    // transposed DC4 along the tangent: cell Y receives
    // sum_o dcw[o] cb(Y - dco[o] e) (dco = -2, -1, 1, 2; dcw = (1, -8, 8, -1) / 12).
    // Slots: x faces (tangent y) 0: du/dy -> u, 1: dv/dy -> v;
    // y faces (tangent x) 2: dv/dx -> v, 3: du/dx -> u.
    for (int t = tid; t < G::ACS; t += G::NT) {
      const int lx = t % G::APX, ly = t / G::APX;
      // (cells beyond the accumulation region hold no cotangent)
      auto spread = [&](int slot, int step, int pos, int len) {
        const T* s = cbuf + slot * G::ACS + t;
        T v = T(0);
        if (pos + 2 < len) v += (T(1) / T(12)) * s[2 * step];
        if (pos + 1 < len) v += (-T(8) / T(12)) * s[step];
        if (pos >= 1) v += (T(8) / T(12)) * s[-step];
        if (pos >= 2) v += (-T(1) / T(12)) * s[-2 * step];
        return v;
      };
      const T du = spread(0, G::APX, ly, G::APY) + spread(3, 1, lx, G::APX);
      const T dv = spread(1, G::APX, ly, G::APY) + spread(2, 1, lx, G::APX);
      acc[G::ACS + t] += du;
      acc[2 * G::ACS + t] += dv;
    }
    __syncthreads();
  }

  {
    // ghost cells of a non-periodic axis pass their cotangents to the cell
    // they copy (if it is in this box); everything else outside the box (and
    // beyond the grid on a periodic axis) belongs to another box, which
    // evaluates the same faces.  Only boxes within reach of such a boundary
    // (or ragged against it) have ghosts to fold; the test is uniform per CTA.
    bool fold = false;
#pragma unroll
    for (int a = 0; a < DIM; ++a) {
      const int B = a == 0 ? BX : BY, h = a == 0 ? G::AX : G::AY;
      fold |= !A.periodic[a] && (g0[a] - h < 0 || g0[a] + B + h > A.n[a]);
    }
    if (fold) {
      for (int t = tid; t < G::ACS; t += G::NT) {
        const int lx = t % G::APX - G::AX, ly = t / G::APX - G::AY;
        const int ox = V.owner(lx, g0[0], A.n[0], A.periodic[0], BX);
        const int oy = DIM >= 2 ? V.owner(ly, g0[1], A.n[1], A.periodic[1], BY) : 0;
        if (ox >= 0 && oy >= 0 && (ox != lx || oy != ly)) {
          const int to = (oy + G::AY) * G::APX + ox + G::AX;
#pragma unroll
          for (int c = 0; c < 6; ++c) atomicAdd(acc + c * G::ACS + to, acc[c * G::ACS + t]);
        }
      }
      __syncthreads();
    }
  }

  // cells: cotangent of W (+T) -> cotangent of U, then the stage combination
  const int tx = tid % BX, ty = tid / BX, tz = 0;
  const int gx = g0[0] + tx, gy = g0[1] + ty;
  if (gx < A.n[0] && gy < A.n[1]) {
    const T r = V.w(0, tx, ty, tz), u = V.w(1, tx, ty, tz), v = V.w(2, tx, ty, tz), w = V.w(3, tx, ty, tz);
    const T p = V.w(4, tx, ty, tz);
    const int cell = (ty + G::AY) * G::APX + tx + G::AX;
    T br = acc[cell], bu = acc[G::ACS + cell], bv = acc[2 * G::ACS + cell], bw = acc[3 * G::ACS + cell];
    T bp = acc[4 * G::ACS + cell];
    const T inv = trcp(r);
    if (VISC) {
      const T bT = acc[5 * G::ACS + cell];
      const T Tc = V.w(5, tx, ty, tz);
      br -= bT * Tc * inv;  // T = p / (rho R)
      bp += bT * Tc * trcp(p);
    }
    T bU[5];
    bU[0] = br - (bu * u + bv * v + bw * w) * inv + bp * g.gm1 * T(0.5) * (u * u + v * v + w * w);
    bU[1] = bu * inv - bp * g.gm1 * u;
    bU[2] = bv * inv - bp * g.gm1 * v;
    bU[3] = bw * inv - bp * g.gm1 * w;
    bU[4] = bp * g.gm1;
    const T dt = T(*A.dt);
    const long long q = (long long)gy * A.n[0] + gx;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      T o = V.m(c, tx, ty, tz) + dt * bU[c];
      if (A.x1) o += A.a1 * A.x1[q + c * A.N];
      if (A.x2) o += A.a2 * A.x2[q + c * A.N];
      A.out[q + c * A.N] = o;
    }
  }
}

}  // namespace jf

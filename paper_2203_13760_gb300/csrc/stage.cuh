// Fused finite-volume RK stage kernel (forward).
//
// One launch evaluates, for every interior cell,
//   out = a Un + b (Us + dt L(Us))            (TVD-RK3 stage, Section 3.2)
// or out = L(Us) (right-hand side only), with L the right-hand side of
// Eq. (FVD): conservative -> primitive conversion (Section 2), WENO5-JS face
// states and HLLC flux (Section 3.3), C4 viscous and heat fluxes (Section
// 3.4), flux divergence (Section 3.1).
//
// Tiling.  A CTA owns a BX x BY column of cells (BX = 32: one warp per row
// of cells).  In 3D it marches along z over a chunk of planes, keeping the
// primitive variables of the planes k-2..k+3 in a six-slot shared-memory ring
// (each plane with a 3-cell x/y halo, edges and corners included, as the
// viscous cross derivatives need them).  Per plane: the new plane k+3 is
// loaded into the slot of plane k-3 (coalesced rows, periodic / zero-gradient
// / slip-wall index map applied per cell, converted to W and T), then the x and y face
// fluxes of plane k are written to shared memory, and each cell thread
// computes the z face k+1/2 of its column, the k-1/2 face kept from the
// previous plane in a per-column shared-memory slot.  Every face flux is
// evaluated once per CTA; only the faces on the tile rim are evaluated twice
// (by both tiles).
//
// Work balance.  The CTA has BY + 1 warps.  x faces: warp w < BY takes face
// row w (faces 0..31), warp BY takes the 33rd face of every row; y faces: warp
// w takes face row w (BY + 1 rows of 32); z faces and cell updates: warps
// 0..BY-1.  Every warp thus computes about the same number of faces between
// two barriers, and each warp reads shared memory row-wise (no bank
// conflicts).  2D and 1D tiles hold one plane and no ring; the row tiles of 2D
// grids (DIM_Y2: one row of BX cells, BX + 32 threads) march along y with the
// ring, their rows as its planes.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <type_traits>

#include "jf_math.cuh"

namespace jf {

constexpr int HALO = 3;

// Kernel dimensionality (template parameter DIM).  1, 2 and 3 are the grid's
// active axes: the tile spans x (1D: one row of BX cells; 2D, 3D: BX x BY
// cells) and, in 3D, marches along z.  DIM_Y2 is a 2D grid whose tile is one
// row of BX cells marching along y: the kernel runs it as the x axis plus a
// marched third axis (its rows as the planes of the march), with the roles of
// y and z, and of the v and w components, exchanged where the state is loaded
// and stored (launch_stage and the batch path remap the grid arguments).
constexpr int DIM_Y2 = 4;
constexpr int plane_dims(int dim) { return dim == 2 || dim == 3 ? 2 : 1; }  // axes spanned by a tile
constexpr bool marches(int dim) { return dim == 3 || dim == DIM_Y2; }      // z-march over planes
constexpr bool axis_on(int dim, int a) {                                   // axis a of the kernel active
  return a == 0 || (a == 1 && plane_dims(dim) == 2) || (a == 2 && marches(dim));
}
// Global component of the kernel's component c (DIM_Y2: v and w exchanged).
constexpr int gcomp(int dim, int c) { return dim == DIM_Y2 && (c == 2 || c == 3) ? 5 - c : c; }

// Bounds-checked debug build (-DJF_DEBUG_BOUNDS): every global and
// shared-memory index of the stage kernels is checked before the access; a
// bad one is printed (at most 32 lines per translation unit) and the access
// is skipped (a load then yields 1), so that the kernel reports the fault
// instead of making it.  Off in the normal build.
#ifdef JF_DEBUG_BOUNDS
static __device__ int jf_debug_lines;
#define JF_CHECK(ok, ...)                                                        \
  ((ok) ? true : ((atomicAdd(&jf_debug_lines, 1) < 32 ? (printf(__VA_ARGS__), 0) : 0), false))
// Trace records in host-mapped memory (they stay readable after a fault):
// slot 0 counts records; record r occupies words 8 + 8 r .. 8 + 8 r + 7.
constexpr int kTraceWords = 1 << 20;
__device__ __forceinline__ void jf_trace(unsigned long long* tr, unsigned long long a, unsigned long long b,
                                         unsigned long long c, unsigned long long d, unsigned long long e,
                                         unsigned long long f, unsigned long long g, unsigned long long h) {
  if (!tr) return;
  const unsigned long long r = atomicAdd(tr, 1ull);
  if (8 + 8 * r + 8 > (unsigned long long)kTraceWords) return;
  volatile unsigned long long* w = tr + 8 + 8 * r;
  w[0] = a; w[1] = b; w[2] = c; w[3] = d; w[4] = e; w[5] = f; w[6] = g; w[7] = h;
  __threadfence_system();
}
unsigned long long* debug_trace_dev();  // host: the trace buffer (allocated at the first call)
#else
#define JF_CHECK(ok, ...) true
#endif

// Per-launch description of one grid and one stage.
template <typename T>
struct StageArgs {
  const T* Us;        // stage input, [5][nz][ny][nx]
  const T* Un;        // U^n for the Shu-Osher combination (read point-wise); null if a == 0
  T* out;             // output, [5][nz][ny][nx]; may equal Un
  const double* dt;   // device scalar (null in right-hand-side mode)
  int nx, ny, nz;
  long long N;        // nx * ny * nz
  int periodic[3];    // 1: periodic axis, 0: zero gradient
  int wall[3];        // slip walls of an axis: bit 0 low side, bit 1 high side
  T inv_h[3];         // 1 / dx_d
  T a, b;             // stage coefficients
  int rhs_only;       // 1: out = L(Us)
  int zchunk;         // planes per CTA along z (3D)
  int* flag;          // device error flag (bit 0: non-physical state)
#ifdef JF_DEBUG_BOUNDS
  unsigned long long* trace;  // host-mapped trace records (debug build)
#endif
};

__device__ __forceinline__ int map_index(int i, int n, int periodic) {
  if (periodic) {
    // one wrap covers the 3-cell halo when n >= 3; the remainder handles
    // shorter periodic axes
    if (i < 0) i += n; else if (i >= n) i -= n;
    if ((unsigned)i >= (unsigned)n) { i %= n; if (i < 0) i += n; }
    return i;
  }
  return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// Index map with slip walls (Table 2 boundary conditions; the extended and
// Rusanov-NN kernel families only): a ghost cell beyond a wall is the mirror
// image of the cell inside (-1 - i at the low side, 2n - 1 - i at the high
// side) and `flip`
// records that its momentum normal to the wall changes sign.  Mirroring each
// axis on its own equals filling the ghost layers axis after axis (edge and
// corner ghosts then carry the product of the flips).  Active axes have at
// least 5 cells, so the mirror of the 3-cell halo stays inside the grid; a
// ragged tile also loads cells further out, which no face uses, and their
// mirror index is clamped into the grid so that every load stays in bounds.
__device__ __forceinline__ int map_index_bc(int i, int n, int periodic, int wall, bool& flip) {
  if (i < 0 && (wall & 1)) { flip = true; return min(-1 - i, n - 1); }
  if (i >= n && (wall & 2)) { flip = true; return max(2 * n - 1 - i, 0); }
  flip = false;
  return map_index(i, n, periodic);
}

// Shared-memory plane geometry.
template <int BX, int BY, int DIM, bool VISC>
struct Geo {
  static constexpr int HY = plane_dims(DIM) == 2 ? HALO : 0;
  static constexpr int PX = BX + 2 * HALO;           // row pitch
  static constexpr int PY = BY + 2 * HY;
  static constexpr int CS = PX * PY;                 // component stride
  static constexpr int NC = VISC ? 6 : 5;            // rho, u, v, w, p (, T)
  static constexpr int PLANE = NC * CS;
  static constexpr int RING = marches(DIM) ? 6 : 1;  // planes held
  static constexpr int NFX = (BX + 1) * BY;          // x faces per plane
  static constexpr int NFY = plane_dims(DIM) == 2 ? BX * (BY + 1) : 0;
  static constexpr int NCELL = BX * BY;              // cell threads
  static constexpr int NT = plane_dims(DIM) == 2 ? BX * (BY + 1) : BX + 32;  // threads
  static_assert(plane_dims(DIM) == 1 || BX == 32, "2D/3D tiles are one warp wide");
  static_assert(plane_dims(DIM) == 2 || BY == 1, "row tiles are one row");
};

// Plane loads are split into a fetch (global loads of the conservative state
// into registers) and a commit (conversion to W (+T) and the shared-memory
// store), so that the fetch of the next plane can be issued before the face
// computations of the current one and its latency overlaps with them.
template <typename T, int BX, int BY, int DIM, bool VISC>
struct PlaneRegs {
  using G = Geo<BX, BY, DIM, VISC>;
  static constexpr int PF = (G::CS + G::NT - 1) / G::NT;  // cells per thread
  T v[PF][5];
};

// Fetch plane gz (global z index, mapped by the boundary condition) of the
// tile at (gx0, gy0).
// WALLS: the kernel handles slip walls (only the extended and Rusanov-NN
// kernel families; the host routes every walled grid to one of them).
template <typename T, int BX, int BY, int DIM, bool VISC, bool WALLS>
__device__ __forceinline__ void fetch_plane(const StageArgs<T>& A, PlaneRegs<T, BX, BY, DIM, VISC>& r, int gx0,
                                            int gy0, int gz) {
  using G = Geo<BX, BY, DIM, VISC>;
  bool fz = false;
  int kz = 0;
  if (marches(DIM)) kz = WALLS ? map_index_bc(gz, A.nz, A.periodic[2], A.wall[2], fz) : map_index(gz, A.nz, A.periodic[2]);
  const long long zoff = (long long)kz * A.ny;
#pragma unroll
  for (int i = 0; i < PlaneRegs<T, BX, BY, DIM, VISC>::PF; ++i) {
    const int t = threadIdx.x + i * G::NT;
    if (t < G::CS) {
      const int ly = t / G::PX;
      const int lx = t - ly * G::PX;
      bool fx = false, fy = false;
      int gx, gy = 0;
      if (WALLS) {
        gx = map_index_bc(gx0 + lx - HALO, A.nx, A.periodic[0], A.wall[0], fx);
        if (plane_dims(DIM) == 2) gy = map_index_bc(gy0 + ly - G::HY, A.ny, A.periodic[1], A.wall[1], fy);
      } else {
        gx = map_index(gx0 + lx - HALO, A.nx, A.periodic[0]);
        if (plane_dims(DIM) == 2) gy = map_index(gy0 + ly - G::HY, A.ny, A.periodic[1]);
      }
      const long long q = (zoff + gy) * A.nx + gx;
#pragma unroll
      for (int c = 0; c < 5; ++c)
        r.v[i][c] = JF_CHECK(q >= 0 && q < A.N, "JFDBG fetch q=%lld N=%lld gx=%d gy=%d kz=%d tile=(%d,%d) t=%d\n", q,
                             A.N, gx, gy, kz, gx0, gy0, t)
                        ? __ldg(A.Us + q + gcomp(DIM, c) * A.N)
                        : T(1);
      if (WALLS) {
        if (fx) r.v[i][1] = -r.v[i][1];
        if (fy) r.v[i][2] = -r.v[i][2];
        if (fz) r.v[i][3] = -r.v[i][3];
      }
    }
  }
}

// In-plane offsets (gy nx + gx, after the index map) of the cells a thread
// fetches: the same for every plane of a z-march without walls, so the march
// computes them once per tile (plane_map) and fetches with them
// (fetch_plane_mapped).
template <typename T, int BX, int BY, int DIM, bool VISC>
struct PlaneMap {
  int off[PlaneRegs<T, BX, BY, DIM, VISC>::PF];
};

template <typename T, int BX, int BY, int DIM, bool VISC>
__device__ __forceinline__ void plane_map(const StageArgs<T>& A, PlaneMap<T, BX, BY, DIM, VISC>& m, int gx0,
                                          int gy0) {
  using G = Geo<BX, BY, DIM, VISC>;
#pragma unroll
  for (int i = 0; i < PlaneRegs<T, BX, BY, DIM, VISC>::PF; ++i) {
    const int t = threadIdx.x + i * G::NT;
    const int ly = t / G::PX, lx = t - ly * G::PX;
    const int gx = map_index(gx0 + lx - HALO, A.nx, A.periodic[0]);
    const int gy = plane_dims(DIM) == 2 ? map_index(gy0 + ly - G::HY, A.ny, A.periodic[1]) : 0;
    m.off[i] = t < G::CS ? gy * A.nx + gx : 0;
  }
}

template <typename T, int BX, int BY, int DIM, bool VISC>
__device__ __forceinline__ void fetch_plane_mapped(const StageArgs<T>& A, PlaneRegs<T, BX, BY, DIM, VISC>& r,
                                                   const PlaneMap<T, BX, BY, DIM, VISC>& m, int gz) {
  using G = Geo<BX, BY, DIM, VISC>;
  const int kz = marches(DIM) ? map_index(gz, A.nz, A.periodic[2]) : 0;
  const long long zoff = (long long)kz * A.ny * A.nx;
#pragma unroll
  for (int i = 0; i < PlaneRegs<T, BX, BY, DIM, VISC>::PF; ++i) {
    const int t = threadIdx.x + i * G::NT;
    if (t < G::CS) {
      const long long q = zoff + m.off[i];
#pragma unroll
      for (int c = 0; c < 5; ++c)
        r.v[i][c] = JF_CHECK(q >= 0 && q < A.N, "JFDBG fetch q=%lld N=%lld t=%d\n", q, A.N, t)
                        ? __ldg(A.Us + q + gcomp(DIM, c) * A.N)
                        : T(1);
    }
  }
}

// Convert fetched conservative values to primitives (+ temperature) and
// store them into the plane at dst.
template <typename T, int BX, int BY, int DIM, bool VISC>
__device__ __forceinline__ void commit_plane(const StageArgs<T>& A, const Gas<T>& g,
                                             const PlaneRegs<T, BX, BY, DIM, VISC>& r, T* dst) {
  using G = Geo<BX, BY, DIM, VISC>;
  bool bad = false;
#pragma unroll
  for (int i = 0; i < PlaneRegs<T, BX, BY, DIM, VISC>::PF; ++i) {
    const int t = threadIdx.x + i * G::NT;
    if (t < G::CS) {
      const T rho = r.v[i][0];
      const T inv = trcp(rho);
      const T u = r.v[i][1] * inv, v = r.v[i][2] * inv, w = r.v[i][3] * inv;
      const T p = g.gm1 * (r.v[i][4] - T(0.5) * rho * (u * u + v * v + w * w));
      bad |= !(rho > T(0)) || !(p > T(0)) || !(p < T(INFINITY));
      dst[t] = rho;
      dst[G::CS + t] = u;
      dst[2 * G::CS + t] = v;
      dst[3 * G::CS + t] = w;
      dst[4 * G::CS + t] = p;
      if (VISC) dst[5 * G::CS + t] = p * inv * g.inv_R;
    }
  }
  if (bad) atomicOr(A.flag, 1);
}

template <typename T, int BX, int BY, int DIM, bool VISC, bool WALLS>
__device__ __forceinline__ void load_plane(const StageArgs<T>& A, const Gas<T>& g, T* dst, int gx0, int gy0,
                                           int gz) {
  PlaneRegs<T, BX, BY, DIM, VISC> r;
  fetch_plane<T, BX, BY, DIM, VISC, WALLS>(A, r, gx0, gy0, gz);
  commit_plane<T, BX, BY, DIM, VISC>(A, g, r, dst);
}

// Accessor of the ring: value of component c at plane offset e (-3..3),
// shared-memory row y, column x (both including the halo offset).
template <typename T, int BX, int BY, int DIM, bool VISC>
struct RingView {
  using G = Geo<BX, BY, DIM, VISC>;
  const T* s;
  int plane[7];  // element offset of plane k + e, index e + 3
  __device__ __forceinline__ T at(int c, int x, int y, int e) const {
    const int i = plane[e + 3] + c * G::CS + y * G::PX + x;
    return JF_CHECK(i >= 0 && i < G::RING * G::PLANE && x >= 0 && x < G::PX && y >= 0 && y < G::PY,
                    "JFDBG ring c=%d x=%d y=%d e=%d i=%d\n", c, x, y, e, i)
               ? s[i]
               : T(1);
  }
};

// Axis roles of a face normal to D: offsets (along normal, tangent 1,
// tangent 2) -> (x, y, plane).
template <int D> struct Roles;
template <> struct Roles<0> {
  static constexpr int T1 = 1, T2 = 2;
  __device__ static void map(int n, int t1, int t2, int& x, int& y, int& e) { x = n; y = t1; e = t2; }
};
template <> struct Roles<1> {
  static constexpr int T1 = 0, T2 = 2;
  __device__ static void map(int n, int t1, int t2, int& x, int& y, int& e) { x = t1; y = n; e = t2; }
};
template <> struct Roles<2> {
  static constexpr int T1 = 0, T2 = 1;
  __device__ static void map(int n, int t1, int t2, int& x, int& y, int& e) { x = t1; y = t2; e = n; }
};

// Scheme codes of the stage kernels (template parameter SCH).
// The _EXT families also handle slip walls and WENO3-JS; their plain
// counterparts leave that code out (it costs the run-time-scheme and ROE
// kernels 15-20 % even on grids without walls: more registers, more spills).
enum { SCH_DEFAULT = 0, SCH_GENERAL = 1, SCH_ROE = 2, SCH_NN = 3, SCH_GENERAL_EXT = 4, SCH_ROE_EXT = 5 };
constexpr bool sch_general(int s) { return s == SCH_GENERAL || s == SCH_GENERAL_EXT; }
constexpr bool sch_roe(int s) { return s == SCH_ROE || s == SCH_ROE_EXT; }
constexpr bool sch_ext(int s) { return s == SCH_GENERAL_EXT || s == SCH_ROE_EXT || s == SCH_NN; }
// Families whose kernels reconstruct once per cell and direction (the face
// values of a plane in shared memory): the default scheme and the run-time
// Godunov schemes with WENO5-JS / WENO5-Z.
constexpr bool sch_pc(int s) { return s == SCH_DEFAULT || s == SCH_GENERAL; }

// Flux-splitting face flux of the ROE setup (Section 3.3, Flux-Splitting
// approach; Section 5): Roe average of the two cells beside the face, the
// eigenvectors of the flux Jacobian there, the six stencil cells' conservative
// states U_j and fluxes F_j projected on the characteristic fields
// (V_j = L U_j, G_j = L F_j), Roe splitting G+-_j = (G_j +- |lambda| V_j) / 2,
// WENO5 of G+ (left-biased, cells -2..2) and G- (mirrored, cells 3..-1) per
// field (WENO3: cells -1..1 and 2..0), and the sum transformed back, F = R (G+ + G-).  L and R are applied
// in closed form (b1 = (gamma - 1) / c^2, b2 = b1 |u|^2 / 2,
// s(X) = b2 X_0 - b1 u.X_m + b1 X_4, d(X) = (u_n X_0 - X_n) / c):
//   L X = [(s + d) / 2, X_0 - s, X_t1 - u_t1 X_0, X_t2 - u_t2 X_0, (s - d) / 2],
//   R G: mass = G0 + G1 + G4 =: S, momentum u S + c n (G4 - G0) + t1 G2 + t2 G3,
//        energy H (G0 + G4) + u_n c (G4 - G0) + |u|^2 / 2 G1 + u_t1 G2 + u_t2 G3.
template <typename T, int D, bool EXT, typename Val>
__device__ __forceinline__ void fs_flux(const Val& val, const Gas<T>& g, int recon, T F[5]) {
  constexpr int T1 = (D + 1) % 3, T2 = (D + 2) % 3;
  // Roe average
  const T rL = val(0, 0), rR = val(0, 1);
  const T sL = tsqrt(rL), sR = tsqrt(rR), is = trcp(sL + sR);
  T u[3];
#pragma unroll
  for (int m = 0; m < 3; ++m) u[m] = (sL * val(1 + m, 0) + sR * val(1 + m, 1)) * is;
  const T kH = g.gamma * g.inv_gm1;  // H = gamma/(gamma-1) p/rho + |u|^2/2
  const T qL = val(1, 0) * val(1, 0) + val(2, 0) * val(2, 0) + val(3, 0) * val(3, 0);
  const T qR = val(1, 1) * val(1, 1) + val(2, 1) * val(2, 1) + val(3, 1) * val(3, 1);
  const T HL = kH * val(4, 0) * trcp(rL) + T(0.5) * qL;
  const T HR = kH * val(4, 1) * trcp(rR) + T(0.5) * qR;
  const T H = (sL * HL + sR * HR) * is;
  const T q2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const T c2 = g.gm1 * (H - T(0.5) * q2);
  const T c = tsqrt(c2), ic = trcp(c);
  const T b1 = g.gm1 * trcp(c2), b2 = T(0.5) * b1 * q2;
  const T un = u[D];
  const T a0 = T(0.5) * fabs(un - c), a1 = T(0.5) * fabs(un), a4 = T(0.5) * fabs(un + c);
  // projected, split fluxes: Pp[k][j] = G+_j (j = 0..4 for cells -2..2),
  // Pm[k][j] = G-_{5-j} (j = 0..4 for cells 3..-1), field k
  T Pp[5][5], Pm[5][5];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const int n = j - 2;
    const T r = val(0, n), v0 = val(1, n), v1 = val(2, n), v2 = val(3, n), p = val(4, n);
    const T vn = D == 0 ? v0 : (D == 1 ? v1 : v2);
    const T E = p * g.inv_gm1 + T(0.5) * r * (v0 * v0 + v1 * v1 + v2 * v2);
    const T U[5] = {r, r * v0, r * v1, r * v2, E};
    const T mass = r * vn;
    T Fj[5] = {mass, mass * v0, mass * v1, mass * v2, vn * (E + p)};
    Fj[1 + D] += p;
    T V[5], G[5];
    auto project = [&](const T X[5], T Y[5]) {
      const T s = b2 * X[0] - b1 * (u[0] * X[1] + u[1] * X[2] + u[2] * X[3]) + b1 * X[4];
      const T d = (un * X[0] - X[1 + D]) * ic;
      Y[0] = T(0.5) * (s + d);
      Y[1] = X[0] - s;
      Y[2] = X[1 + T1] - u[T1] * X[0];
      Y[3] = X[1 + T2] - u[T2] * X[0];
      Y[4] = T(0.5) * (s - d);
    };
    project(U, V);
    project(Fj, G);
    const T a[5] = {a0, a1, a1, a1, a4};
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const T half_g = T(0.5) * G[k];
      if (j <= 4) Pp[k][j] = half_g + a[k] * V[k];
      if (j >= 1) Pm[k][5 - j] = half_g - a[k] * V[k];
    }
  }
  T Gh[5];
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    if (EXT && recon == 2) {  // WENO3-JS: G+ from cells -1..1, G- from cells 2..0
      if constexpr (sizeof(T) == 4) {
        const float2 r = weno3_pair(make_float2(Pp[k][1], Pm[k][1]), make_float2(Pp[k][2], Pm[k][2]),
                                    make_float2(Pp[k][3], Pm[k][3]), g.eps);
        Gh[k] = r.x + r.y;
      } else {
        Gh[k] = weno3(Pp[k][1], Pp[k][2], Pp[k][3], g.eps) + weno3(Pm[k][1], Pm[k][2], Pm[k][3], g.eps);
      }
      continue;
    }
    if constexpr (sizeof(T) == 4) {
      const float2 r = weno5_pair(make_float2(Pp[k][0], Pm[k][0]), make_float2(Pp[k][1], Pm[k][1]),
                                  make_float2(Pp[k][2], Pm[k][2]), make_float2(Pp[k][3], Pm[k][3]),
                                  make_float2(Pp[k][4], Pm[k][4]), g.eps, recon);
      Gh[k] = r.x + r.y;
    } else {
      Gh[k] = weno5(Pp[k][0], Pp[k][1], Pp[k][2], Pp[k][3], Pp[k][4], g.eps, recon) +
              weno5(Pm[k][0], Pm[k][1], Pm[k][2], Pm[k][3], Pm[k][4], g.eps, recon);
    }
  }
  const T S = Gh[0] + Gh[1] + Gh[4], Dw = Gh[4] - Gh[0];
  F[0] = S;
  F[1 + D] = u[D] * S + c * Dw;
  F[1 + T1] = u[T1] * S + Gh[2];
  F[1 + T2] = u[T2] * S + Gh[3];
  F[4] = H * (Gh[0] + Gh[4]) + un * c * Dw + T(0.5) * q2 * Gh[1] + u[T1] * Gh[2] + u[T2] * Gh[3];
}

// Convective flux F of a Godunov-type face from its reconstructed states Wm
// (left) and Wp (right): the safe-reconstruction fallback, then the Riemann
// solver of the kernel family.
template <typename T, int D, int BX, int BY, int DIM, bool VISC, int SCH>
__device__ __forceinline__ void face_riemann(const RingView<T, BX, BY, DIM, VISC>& R, int x0, int y0,
                                             const Gas<T>& g, T Wm[5], T Wp[5], T F[5]) {
  using Ro = Roles<D>;
  auto val = [&](int c, int n, int t1, int t2) -> T {
    int x, y, e;
    Ro::map(n, t1, t2, x, y, e);
    return R.at(c, x0 + x, y0 + y, e);
  };
  if (g.safe) {
    if (!(Wm[0] > T(0)) || !(Wm[4] > T(0))) {
#pragma unroll
      for (int c = 0; c < 5; ++c) Wm[c] = val(c, 0, 0, 0);
    }
    if (!(Wp[0] > T(0)) || !(Wp[4] > T(0))) {
#pragma unroll
      for (int c = 0; c < 5; ++c) Wp[c] = val(c, 1, 0, 0);
    }
  }
  if constexpr (sch_general(SCH)) riemann_flux<T, D>(Wm, Wp, g, F);
  else if constexpr (SCH == SCH_NN) rusanov_nn<T, D>(Wm, Wp, g, F);
  else hllc<T, D>(Wm, Wp, g, F, 0);
}

// Cell-centre C4 tangential derivative sums of the z faces of one column
// (FP32, z-marching kernels): h[t][j] for tangent t (0: x, 1: y) at the
// planes k, k + 1, k + 2 of the face k + 1/2 (j = 0, 1, 2), the packed pair
// (w, u_t) as in face_visc_add.  The face k + 3/2 reuses them and computes
// only plane k + 3.
struct ZTangents {
  float2 h[2][3];
};

// Dissipative part of the net flux (Sections 2 and 3.4) through the face
// between the cell at shared-memory position (x0, y0, plane 0) and its
// neighbour along D, added to NF.
// ZC (FP32, D == 2 only): 0 computes every tangential stencil; 1 computes
// them and keeps those of planes 0..2 in *zc; 2 takes planes -1..1 from *zc,
// computes plane 2 and shifts *zc to planes 0..2.
template <typename T, int D, int BX, int BY, int DIM, bool VISC, int ZC = 0>
__device__ __forceinline__ void face_visc_add(const RingView<T, BX, BY, DIM, VISC>& R, int x0, int y0,
                                              const Gas<T>& g, const T inv_h[3], T NF[5],
                                              ZTangents* zc = nullptr) {
  static_assert(ZC == 0 || (D == 2 && sizeof(T) == 4), "carried tangential stencils: FP32 z faces only");
  using Ro = Roles<D>;
  auto val = [&](int c, int n, int t1, int t2) -> T {
    int x, y, e;
    Ro::map(n, t1, t2, x, y, e);
    return R.at(c, x0 + x, y0 + y, e);
  };
  // Dissipative flux (Sections 2 and 3.4).  G[a][b] = du_a/dx_b at the face.
  T G[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) G[a][b] = T(0);
  const T hn = inv_h[D];
  T dTdn, uf[3];
  if constexpr (sizeof(T) == 4) {
    // FP32: the same stencils on component pairs in packed FP32x2 arithmetic
    // (equal to the scalar form below up to rounding)
    auto c2 = [](float x) { return make_float2(x, x); };
    const float2 m1 = c2(-1.0f);
    auto pair = [&](int c0, int c1, int n, int t1, int t2) {
      return make_float2(val(c0, n, t1, t2), val(c1, n, t1, t2));
    };
    // normal derivative (df4) and face value (rc4) from the cells -1..2
    // along the normal: (u, v) and (w, T)
    float2 uv[4], wT[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uv[q] = pair(1, 2, q - 1, 0, 0);
      wT[q] = pair(3, 5, q - 1, 0, 0);
    }
    const float2 kn27 = c2(27.0f / 24.0f * hn), kn1 = c2(hn / 24.0f);
    auto df4p = [&](const float2 v[4]) {
      return __ffma2_rn(kn27, __ffma2_rn(m1, v[1], v[2]), __fmul2_rn(kn1, __ffma2_rn(m1, v[3], v[0])));
    };
    auto rc4p = [&](const float2 v[4]) {
      return __ffma2_rn(c2(9.0f / 16.0f), __fadd2_rn(v[1], v[2]), __fmul2_rn(c2(-1.0f / 16.0f), __fadd2_rn(v[0], v[3])));
    };
    const float2 g_uv = df4p(uv), g_wT = df4p(wT), f_uv = rc4p(uv), f_wT = rc4p(wT);
    G[0][D] = g_uv.x;
    G[1][D] = g_uv.y;
    G[2][D] = g_wT.x;
    dTdn = g_wT.y;
    uf[0] = f_uv.x;
    uf[1] = f_uv.y;
    uf[2] = f_wT.x;
    // tangential derivative along e of (u_D, u_e): cell-centre C4 derivative
    // at the cells -1..2 along the normal, interpolated to the face:
    // h_q = (v(q,-2) - v(q,2)) + 8 (v(q,1) - v(q,-1)), G = (9 (h1 + h2) - (h0 + h3)) / 192
    auto tang = [&](auto role) {
      constexpr int R = decltype(role)::value;  // 1: tangent T1, 2: tangent T2
      constexpr int e = R == 1 ? Ro::T1 : Ro::T2;
      float2 h[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (ZC == 2 && q < 3) {
          h[q] = zc->h[R - 1][q];
          continue;
        }
        auto at = [&](int j) { return R == 1 ? pair(1 + D, 1 + e, q - 1, j, 0) : pair(1 + D, 1 + e, q - 1, 0, j); };
        const float2 vm2 = at(-2), vm1 = at(-1), vp1 = at(1), vp2 = at(2);
        h[q] = __ffma2_rn(c2(8.0f), __ffma2_rn(m1, vm1, vp1), __ffma2_rn(m1, vp2, vm2));
      }
      if (ZC != 0) {
#pragma unroll
        for (int q = 0; q < 3; ++q) zc->h[R - 1][q] = h[q + 1];
      }
      const float he = inv_h[e];
      const float2 Ge = __ffma2_rn(c2(9.0f / 192.0f * he), __fadd2_rn(h[1], h[2]),
                                   __fmul2_rn(c2(-1.0f / 192.0f * he), __fadd2_rn(h[0], h[3])));
      G[D][e] = Ge.x;
      G[e][e] = Ge.y;
    };
    if constexpr (axis_on(DIM, Ro::T1)) tang(std::integral_constant<int, 1>{});
    if constexpr (axis_on(DIM, Ro::T2)) tang(std::integral_constant<int, 2>{});
  } else {
#pragma unroll
  for (int a = 0; a < 3; ++a)
    G[a][D] = df4(val(1 + a, -1, 0, 0), val(1 + a, 0, 0, 0), val(1 + a, 1, 0, 0), val(1 + a, 2, 0, 0)) * hn;
  dTdn = df4(val(5, -1, 0, 0), val(5, 0, 0, 0), val(5, 1, 0, 0), val(5, 2, 0, 0)) * hn;
  // tangential derivatives: cell-centre C4 at cells -1..2 along the normal,
  // then fourth-order interpolation to the face
  if (axis_on(DIM, Ro::T1)) {
    constexpr int e = Ro::T1;
    const T he = inv_h[e];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int a = s == 0 ? D : e;
      T cen[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        cen[q] = dc4(val(1 + a, q - 1, -2, 0), val(1 + a, q - 1, -1, 0), val(1 + a, q - 1, 1, 0),
                     val(1 + a, q - 1, 2, 0));
      G[a][e] = rc4(cen[0], cen[1], cen[2], cen[3]) * he;
    }
  }
  if (axis_on(DIM, Ro::T2)) {
    constexpr int e = Ro::T2;
    const T he = inv_h[e];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int a = s == 0 ? D : e;
      T cen[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        cen[q] = dc4(val(1 + a, q - 1, 0, -2), val(1 + a, q - 1, 0, -1), val(1 + a, q - 1, 0, 1),
                     val(1 + a, q - 1, 0, 2));
      G[a][e] = rc4(cen[0], cen[1], cen[2], cen[3]) * he;
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a)
    uf[a] = rc4(val(1 + a, -1, 0, 0), val(1 + a, 0, 0, 0), val(1 + a, 1, 0, 0), val(1 + a, 2, 0, 0));
  }
  const T div = G[0][0] + G[1][1] + G[2][2];
  T tau[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) tau[a] = g.mu * (G[D][a] + G[a][D]);
  tau[D] -= (T(2) / T(3)) * g.mu * div;
  NF[1] += tau[0];
  NF[2] += tau[1];
  NF[3] += tau[2];
  NF[4] += uf[0] * tau[0] + uf[1] * tau[1] + uf[2] * tau[2] + g.lambda * dTdn;
}

// Net flux NF = F^d - F through the face between the cell at shared-memory
// position (x0, y0, plane 0) and its neighbour along D.
// SCH_DEFAULT: the default scheme (WENO5-JS, HLLC, Einfeldt speeds) compiled
// alone; SCH_GENERAL(_EXT): the Table 2 Godunov variants chosen at run time
// from g; SCH_ROE(_EXT): the flux-splitting ROE setup (reconstruction chosen
// from g); the _EXT forms add WENO3-JS (and walls, in the plane fetch);
// SCH_NN: the Rusanov-NN flux (Section 7.4; reconstruction chosen from g),
// a kernel family of its own because the network's hidden layers need far
// more registers than the other fluxes.
template <typename T, int D, int BX, int BY, int DIM, bool VISC, int SCH>
__device__ __forceinline__ void face_flux(const RingView<T, BX, BY, DIM, VISC>& R, int x0, int y0,
                                          const Gas<T>& g, const T inv_h[3], T NF[5]) {
  using Ro = Roles<D>;
  const int recon = SCH == SCH_DEFAULT ? 0 : g.recon;
  auto val = [&](int c, int n, int t1, int t2) -> T {
    int x, y, e;
    Ro::map(n, t1, t2, x, y, e);
    return R.at(c, x0 + x, y0 + y, e);
  };
  T F[5];
  if constexpr (sch_roe(SCH)) {
    fs_flux<T, D, sch_ext(SCH)>([&](int c, int n) { return val(c, n, 0, 0); }, g, recon, F);
  } else {
  // WENO5-JS left / right states of each primitive component (Section 3.3)
  T Wm[5], Wp[5];
  if (sch_ext(SCH) && recon == 2) {
    // WENO3-JS: cells -1, 0, 1 (left state) and 2, 1, 0 (right state)
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      const T v1 = val(c, -1, 0, 0), v2 = val(c, 0, 0, 0), v3 = val(c, 1, 0, 0), v4 = val(c, 2, 0, 0);
      if constexpr (sizeof(T) == 4) {
        const float2 r = weno3_pair(make_float2(v1, v4), make_float2(v2, v3), make_float2(v3, v2), g.eps);
        Wm[c] = r.x;
        Wp[c] = r.y;
      } else {
        Wm[c] = weno3(v1, v2, v3, g.eps);
        Wp[c] = weno3(v4, v3, v2, g.eps);
      }
    }
  } else {
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    const T v0 = val(c, -2, 0, 0), v1 = val(c, -1, 0, 0), v2 = val(c, 0, 0, 0);
    const T v3 = val(c, 1, 0, 0), v4 = val(c, 2, 0, 0), v5 = val(c, 3, 0, 0);
    if constexpr (sizeof(T) == 4) {
      const float2 r = weno5_pair(make_float2(v0, v5), make_float2(v1, v4), make_float2(v2, v3), make_float2(v3, v2),
                                  make_float2(v4, v1), g.eps, recon);
      Wm[c] = r.x;
      Wp[c] = r.y;
    } else {
      Wm[c] = weno5(v0, v1, v2, v3, v4, g.eps, recon);
      Wp[c] = weno5(v5, v4, v3, v2, v1, g.eps, recon);
    }
  }
  }
  face_riemann<T, D, BX, BY, DIM, VISC, SCH>(R, x0, y0, g, Wm, Wp, F);
  }
#pragma unroll
  for (int c = 0; c < 5; ++c) NF[c] = -F[c];
  if constexpr (VISC) face_visc_add<T, D, BX, BY, DIM, VISC>(R, x0, y0, g, inv_h, NF);
}

// WENO5 face values of one cell along D (per-cell families, weno5_cell; z:
// the WENO5-Z weights): the cell sits `shift` cells along D from ring
// position (x0, y0, plane 0);
// right[c] = v^-_{+1/2}, its value at the face to its right (the left state
// of that face), left[c] = v^+_{-1/2} (the right state of the face to its
// left).  FP32: (rho, p) and (u, v) in packed lanes, w alone (or, NOW, not
// at all: the caller pairs it with another cell's w).
template <typename T, int D, int BX, int BY, int DIM, bool VISC, bool NOW = false>
__device__ __forceinline__ void cell_recon(const RingView<T, BX, BY, DIM, VISC>& R, int x0, int y0, int shift, T eps,
                                           T right[5], T left[5], int z = 0) {
  using Ro = Roles<D>;
  auto val = [&](int c, int n) -> T {
    int x, y, e;
    Ro::map(n + shift, 0, 0, x, y, e);
    return R.at(c, x0 + x, y0 + y, e);
  };
  if constexpr (sizeof(T) == 4) {
    auto pr = [&](int a, int b, int n) { return make_float2(val(a, n), val(b, n)); };
    float2 r, l;
    weno5_cell_pair(pr(0, 4, -2), pr(0, 4, -1), pr(0, 4, 0), pr(0, 4, 1), pr(0, 4, 2), eps, r, l, z);
    right[0] = r.x; right[4] = r.y; left[0] = l.x; left[4] = l.y;
    weno5_cell_pair(pr(1, 2, -2), pr(1, 2, -1), pr(1, 2, 0), pr(1, 2, 1), pr(1, 2, 2), eps, r, l, z);
    right[1] = r.x; right[2] = r.y; left[1] = l.x; left[2] = l.y;
    if constexpr (!NOW)
      weno5_cell<float>(val(3, -2), val(3, -1), val(3, 0), val(3, 1), val(3, 2), eps, right[3], left[3], z);
  } else {
#pragma unroll
    for (int c = 0; c < 5; ++c)
      weno5_cell<T>(val(c, -2), val(c, -1), val(c, 0), val(c, 1), val(c, 2), eps, right[c], left[c], z);
  }
}

// The stage kernel.  blockDim.x == Geo::NT.
// grid = (ceil(nx/BX), ceil(ny/BY), ceil(nz/zchunk)) (3D), (.., .., 1) otherwise.
// One tile (tile column (bx, by), z chunk bz) of one grid: the whole stage
// for its cells.  Shared memory: the ring and the face buffers.  All threads
// of the CTA call it; it starts and ends without pending shared-memory reads
// that a following call could disturb (the first barrier inside orders them).
template <typename T, int DIM, bool VISC, int BX, int BY, int SCH>
__device__ __forceinline__ void stage_tile(const StageArgs<T>& A, const Gas<T>& g, int bx, int by, int bz,
                                           T* smem) {
  using G = Geo<BX, BY, DIM, VISC>;
  constexpr bool WALLS = sch_ext(SCH);
  T* ring = smem;
  T* Fx = ring + G::RING * G::PLANE;      // [5][BY][BX+1]
  T* Fy = Fx + 5 * G::NFX;                // [5][BY+1][BX]

  const int gx0 = bx * BX;
  const int gy0 = by * BY;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool cell_thread = threadIdx.x < G::NCELL;
  const int tx = threadIdx.x % BX;
  const int ty = threadIdx.x / BX;
  const int gx = gx0 + tx, gy = gy0 + ty;
  const bool own = cell_thread && gx < A.nx && gy < A.ny;
  const T dt = A.rhs_only ? T(0) : T(*A.dt);
  const T inv_h[3] = {A.inv_h[0], A.inv_h[1], A.inv_h[2]};

  // this thread's x face (-1: none) and y face, as (column, row) in the tile
  int xf_x = -1, xf_y = 0;
  if (plane_dims(DIM) == 1) {
    if (threadIdx.x <= BX) { xf_x = threadIdx.x; xf_y = 0; }
  } else if (warp < BY) {
    xf_x = lane; xf_y = warp;
  } else if (lane < BY) {
    xf_x = BX; xf_y = lane;
  }
  const int yf_x = lane, yf_y = warp;  // tiles spanning y: NT == BX * (BY + 1) y faces

  int z0 = 0, z1 = 1;
  if (marches(DIM)) {
    z0 = bz * A.zchunk;
    z1 = min(z0 + A.zchunk, A.nz);
  }

  RingView<T, BX, BY, DIM, VISC> R;
  R.s = ring;
  // plane p lives in slot (p - z0 + 3) mod 6; set_view(b) maps plane offset
  // e (-3..3) of the current plane to slot (b + e + 3) mod 6, b being the
  // slot of plane (current - 3)
  auto set_view = [&](int b) {
#pragma unroll
    for (int e = 0; e < 7; ++e) {
      int s = b + e;
      s = s >= G::RING ? s - G::RING : s;
      s = s >= G::RING ? s - G::RING : s;
      R.plane[e] = (marches(DIM) ? s : 0) * G::PLANE;
    }
  };

  // per-cell families (sch_pc): WENO5 runs once per cell and direction (weno5_cell), the
  // face values of a plane kept in shared memory (x, y; along z only the
  // current cell's value at its upper face, zl, is kept, by its column)
  constexpr bool PC = sch_pc(SCH);
  const int wz = SCH == SCH_DEFAULT ? 0 : g.recon;  // per-cell WENO5: 0 JS, 1 Z
  constexpr int SX = BY * (BX + 2), SY = plane_dims(DIM) == 2 ? (BY + 2) * BX : 0;
  T* EX = Fy + 5 * G::NFY;  // [2][5][BY][BX+2] (PC only)
  T* EY = EX + 2 * 5 * SX;  // [2][5][BY+2][BX] (PC, tiles spanning y)
  // per-cell families, 3D: the net fluxes of a column's z faces in shared
  // memory, [2][5][NCELL] (face k + 1/2 in slot k & 1), written and read by
  // the column's own thread, so that they hold no registers across the phases
  constexpr bool ZS = PC && marches(DIM);
  T* ZF = EY + 2 * 5 * SY;
  auto zf = [&](int k, int c) -> T& { return ZF[((k & 1) * 5 + c) * G::NCELL + threadIdx.x]; };
  // and the WENO5 value of the column's cell k at k + 1/2 (the left state of
  // the next z face), [5][NCELL]
  auto zl = [&](int c) -> T& { return ZF[(10 + c) * G::NCELL + threadIdx.x]; };
  T NFz_lo[5] = {T(0), T(0), T(0), T(0), T(0)};  // other schemes: the lower z face's net flux
  ZTangents ztan;  // FP32 z faces: the tangential stencils of the planes k .. k + 2
  PlaneRegs<T, BX, BY, DIM, VISC> next;  // plane k + 4, in flight while plane k is computed
  PlaneMap<T, BX, BY, DIM, VISC> pmap;    // per-cell families (no walls): the in-plane offsets of its cells
  if constexpr (PC && marches(DIM)) plane_map<T, BX, BY, DIM, VISC>(A, pmap, gx0, gy0);
  if (marches(DIM)) {
#pragma unroll 1
    for (int q = 0; q < 6; ++q) load_plane<T, BX, BY, DIM, VISC, WALLS>(A, g, ring + q * G::PLANE, gx0, gy0, z0 - 3 + q);
    __syncthreads();
    // lower face of plane z0 = upper face of plane z0 - 1 (slot 2); plane
    // offset -3 is never read
    set_view(5);
    if (cell_thread) {
      if constexpr (PC) {
        // face z0 - 1/2 from the values of cells z0 - 1 and z0; zl: cell z0 at z0 + 1/2
        T r[5], l[5], rz[5], lz[5];
        cell_recon<T, 2, BX, BY, DIM, VISC>(R, HALO + tx, G::HY + ty, 0, g.eps, r, l, wz);
        cell_recon<T, 2, BX, BY, DIM, VISC>(R, HALO + tx, G::HY + ty, 1, g.eps, rz, lz, wz);
#pragma unroll
        for (int c = 0; c < 5; ++c) zl(c) = rz[c];
        T F[5], NF[5];
        face_riemann<T, 2, BX, BY, DIM, VISC, SCH>(R, HALO + tx, G::HY + ty, g, r, lz, F);
#pragma unroll
        for (int c = 0; c < 5; ++c) NF[c] = -F[c];
        if constexpr (VISC && sizeof(T) == 4)
          face_visc_add<T, 2, BX, BY, DIM, VISC, 1>(R, HALO + tx, G::HY + ty, g, inv_h, NF, &ztan);
        else if constexpr (VISC)
          face_visc_add<T, 2, BX, BY, DIM, VISC>(R, HALO + tx, G::HY + ty, g, inv_h, NF);
#pragma unroll
        for (int c = 0; c < 5; ++c) zf(z0 - 1, c) = NF[c];
      } else {
        face_flux<T, 2, BX, BY, DIM, VISC, SCH>(R, HALO + tx, G::HY + ty, g, inv_h, NFz_lo);
      }
    }
    __syncthreads();  // slot 0 (plane z0 - 3) is overwritten next
    load_plane<T, BX, BY, DIM, VISC, WALLS>(A, g, ring, gx0, gy0, z0 + 3);
    // (per-cell families: each plane fetches plane k + 4 after its reconstruction phase)
    if (!PC && z0 + 1 < z1) fetch_plane<T, BX, BY, DIM, VISC, WALLS>(A, next, gx0, gy0, z0 + 4);
  } else {
    load_plane<T, BX, BY, DIM, VISC, WALLS>(A, g, ring, gx0, gy0, 0);
  }
  __syncthreads();

  int base = 0;  // slot of plane k - 3 (and of plane k + 3)
  for (int k = z0; k < z1; ++k) {
    set_view(base);
    // this cell's U_s and U^n for the stage combination, loaded ahead of the
    // face computations so that their latency overlaps with them (per-cell
    // families in 3D: after the x face, which keeps their registers free during
    // the reconstruction phase and the x face; the 3D march holds more state)
    const long long qc = ((long long)(marches(DIM) ? k : 0) * A.ny + gy) * A.nx + gx;
    T us[5], un[5];
    auto load_cell = [&]() {
      if (own && !A.rhs_only) {
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          const bool ok = JF_CHECK(qc >= 0 && qc < A.N, "JFDBG cell qc=%lld N=%lld\n", qc, A.N);
          us[c] = ok ? __ldg(A.Us + qc + gcomp(DIM, c) * A.N) : T(1);
          un[c] = A.Un && ok ? A.Un[qc + gcomp(DIM, c) * A.N] : T(0);
        }
      }
    };
    // (per-cell families in 3D: after the x face below)
    if constexpr (!PC || DIM != 3) load_cell();

    T NFz_hi[5];
    if constexpr (PC) {
      // phase 1: face values of the cells along x (rows 0 .. BY-1, cells
      // -1 .. BX) and y (rows -1 .. BY), and the z face of each column
      auto put_x = [&](int row, int j) {
        T r[5], l[5];
        cell_recon<T, 0, BX, BY, DIM, VISC>(R, HALO + j, G::HY + row, 0, g.eps, r, l, wz);
        const int i = row * (BX + 2) + j + 1;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          if (JF_CHECK(i >= 0 && i < SX, "JFDBG EX i=%d\n", i)) {
            EX[c * SX + i] = r[c];
            EX[(5 + c) * SX + i] = l[c];
          }
        }
      };
      auto put_y = [&](int row, int x) {
        T r[5], l[5];
        cell_recon<T, 1, BX, BY, DIM, VISC>(R, HALO + x, G::HY + row, 0, g.eps, r, l, wz);
        const int i = (row + 1) * BX + x;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          if (JF_CHECK(i >= 0 && i < SY, "JFDBG EY i=%d\n", i)) {
            EY[c * SY + i] = r[c];
            EY[(5 + c) * SY + i] = l[c];
          }
        }
      };
      if (plane_dims(DIM) == 1) {
        if (threadIdx.x < BX + 2) put_x(0, (int)threadIdx.x - 1);
      } else if constexpr (sizeof(T) == 4) {
        // the same cells as below; the w components of a thread's x cell and
        // (first) y cell share one packed WENO5 (threads without an x cell
        // reconstruct an in-range one and discard it)
        const bool hx = warp < BY || lane < 2 * BY;
        const int xrow = warp < BY ? warp : (hx ? lane >> 1 : 0);
        const int xcol = warp < BY ? lane - 1 : (hx ? BX - 1 + (lane & 1) : 0);
        const int yrow0 = warp < BY ? warp - 1 : BY - 1;
        T r[5], l[5];
        cell_recon<T, 0, BX, BY, DIM, VISC, true>(R, HALO + xcol, G::HY + xrow, 0, g.eps, r, l, wz);
        const int ix = xrow * (BX + 2) + xcol + 1;
        if (hx) {
#pragma unroll
          for (int c = 0; c < 5; ++c) {
            if (c == 3) continue;
            if (JF_CHECK(ix >= 0 && ix < SX, "JFDBG EX i=%d\n", ix)) {
              EX[c * SX + ix] = r[c];
              EX[(5 + c) * SX + ix] = l[c];
            }
          }
        }
        cell_recon<T, 1, BX, BY, DIM, VISC, true>(R, HALO + lane, G::HY + yrow0, 0, g.eps, r, l, wz);
        const int iy = (yrow0 + 1) * BX + lane;
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          if (c == 3) continue;
          if (JF_CHECK(iy >= 0 && iy < SY, "JFDBG EY i=%d\n", iy)) {
            EY[c * SY + iy] = r[c];
            EY[(5 + c) * SY + iy] = l[c];
          }
        }
        float2 wv[5];
#pragma unroll
        for (int n = 0; n < 5; ++n)
          wv[n] = make_float2(R.at(3, HALO + xcol + n - 2, G::HY + xrow, 0), R.at(3, HALO + lane, G::HY + yrow0 + n - 2, 0));
        float2 wr, wl;
        weno5_cell_pair(wv[0], wv[1], wv[2], wv[3], wv[4], g.eps, wr, wl, wz);
        if (hx && JF_CHECK(ix >= 0 && ix < SX, "JFDBG EX i=%d\n", ix)) {
          EX[3 * SX + ix] = wr.x;
          EX[8 * SX + ix] = wl.x;
        }
        if (JF_CHECK(iy >= 0 && iy < SY, "JFDBG EY i=%d\n", iy)) {
          EY[3 * SY + iy] = wr.y;
          EY[8 * SY + iy] = wl.y;
        }
        if (warp == BY) put_y(BY, lane);  // warp BY's second y row
      } else {
        // warps 0 .. BY-1: x row `warp` (cells -1 .. 30), y row warp - 1;
        // warp BY: cells 31, 32 of every x row and the y rows BY - 1, BY.
        // One call site each (the loop is not unrolled), so that the code of
        // the plane loop stays small for the instruction cache.
        const int xrow = warp < BY ? warp : (lane < 2 * BY ? lane >> 1 : -1);
        const int xcol = warp < BY ? lane - 1 : BX - 1 + (lane & 1);
        if (xrow >= 0) put_x(xrow, xcol);
        const int yrow0 = warp < BY ? warp - 1 : BY - 1, nyrows = warp < BY ? 1 : 2;
#pragma unroll 1
        for (int q = 0; q < nyrows; ++q) put_y(yrow0 + q, lane);
      }
      if (marches(DIM) && cell_thread) {
        // face k + 1/2: the stored value of cell k (zl) and the lower value of cell k + 1
        T r[5], l[5], F[5], NF[5], zl0[5];
        cell_recon<T, 2, BX, BY, DIM, VISC>(R, HALO + tx, G::HY + ty, 1, g.eps, r, l, wz);
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          zl0[c] = zl(c);
          zl(c) = r[c];
        }
        face_riemann<T, 2, BX, BY, DIM, VISC, SCH>(R, HALO + tx, G::HY + ty, g, zl0, l, F);
#pragma unroll
        for (int c = 0; c < 5; ++c) NF[c] = -F[c];
        if constexpr (VISC && sizeof(T) == 4)
          face_visc_add<T, 2, BX, BY, DIM, VISC, 2>(R, HALO + tx, G::HY + ty, g, inv_h, NF, &ztan);
        else if constexpr (VISC)
          face_visc_add<T, 2, BX, BY, DIM, VISC>(R, HALO + tx, G::HY + ty, g, inv_h, NF);
#pragma unroll
        for (int c = 0; c < 5; ++c) zf(k, c) = NF[c];
      }
      __syncthreads();
      // plane k + 4 in flight during the faces and the update (committed at
      // the end of this plane); its registers are free during the
      // reconstruction phase
      if (marches(DIM) && k + 1 < z1) fetch_plane_mapped<T, BX, BY, DIM, VISC>(A, next, pmap, k + 4);
      // phase 2: the x and y faces from the stored values
      if (xf_x >= 0) {
        T Wm[5], Wp[5], F[5], NF[5];
        const int i = xf_y * (BX + 2) + xf_x;  // left cell xf_x - 1
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          Wm[c] = EX[c * SX + i];
          Wp[c] = EX[(5 + c) * SX + i + 1];
        }
        face_riemann<T, 0, BX, BY, DIM, VISC, SCH>(R, HALO + xf_x - 1, G::HY + xf_y, g, Wm, Wp, F);
#pragma unroll
        for (int c = 0; c < 5; ++c) NF[c] = -F[c];
        if constexpr (VISC) face_visc_add<T, 0, BX, BY, DIM, VISC>(R, HALO + xf_x - 1, G::HY + xf_y, g, inv_h, NF);
        const int t = xf_y * (BX + 1) + xf_x;
#pragma unroll
        for (int c = 0; c < 5; ++c)
          if (JF_CHECK(t >= 0 && t < G::NFX, "JFDBG Fx t=%d\n", t)) Fx[c * G::NFX + t] = NF[c];
      }
      if constexpr (DIM == 3) load_cell();
      if (plane_dims(DIM) == 2) {
        T Wm[5], Wp[5], F[5], NF[5];
        const int i = yf_y * BX + yf_x;  // lower cell row yf_y - 1
#pragma unroll
        for (int c = 0; c < 5; ++c) {
          Wm[c] = EY[c * SY + i];
          Wp[c] = EY[(5 + c) * SY + i + BX];
        }
        face_riemann<T, 1, BX, BY, DIM, VISC, SCH>(R, HALO + yf_x, G::HY + yf_y - 1, g, Wm, Wp, F);
#pragma unroll
        for (int c = 0; c < 5; ++c) NF[c] = -F[c];
        if constexpr (VISC) face_visc_add<T, 1, BX, BY, DIM, VISC>(R, HALO + yf_x, G::HY + yf_y - 1, g, inv_h, NF);
        const int t = yf_y * BX + yf_x;
#pragma unroll
        for (int c = 0; c < 5; ++c)
          if (JF_CHECK(t >= 0 && t < G::NFY, "JFDBG Fy t=%d\n", t)) Fy[c * G::NFY + t] = NF[c];
      }
    } else {
    if (xf_x >= 0) {
      T NF[5];
      face_flux<T, 0, BX, BY, DIM, VISC, SCH>(R, HALO + xf_x - 1, G::HY + xf_y, g, inv_h, NF);
      const int t = xf_y * (BX + 1) + xf_x;
#pragma unroll
      for (int c = 0; c < 5; ++c)
        if (JF_CHECK(t >= 0 && t < G::NFX, "JFDBG Fx t=%d\n", t)) Fx[c * G::NFX + t] = NF[c];
    }
    if (plane_dims(DIM) == 2) {
      T NF[5];
      face_flux<T, 1, BX, BY, DIM, VISC, SCH>(R, HALO + yf_x, G::HY + yf_y - 1, g, inv_h, NF);
      const int t = yf_y * BX + yf_x;
#pragma unroll
      for (int c = 0; c < 5; ++c)
        if (JF_CHECK(t >= 0 && t < G::NFY, "JFDBG Fy t=%d\n", t)) Fy[c * G::NFY + t] = NF[c];
    }
    if (marches(DIM) && cell_thread) face_flux<T, 2, BX, BY, DIM, VISC, SCH>(R, HALO + tx, G::HY + ty, g, inv_h, NFz_hi);
    }
    __syncthreads();

    if constexpr (sizeof(T) == 4 && (ZS || !marches(DIM))) {
      // FP32: the components (0, 1) and (2, 3) in the lanes of packed
      // operations (per lane the operations of the scalar form below), 4 alone
      if (own) {
        const int fx = ty * (BX + 1) + tx, fy = ty * BX + tx;
        const float2 m1 = make_float2(-1.0f, -1.0f);
        auto c2 = [](float x) { return make_float2(x, x); };
        auto comb = [&](int c, bool two) {  // components c and (two) c + 1
          auto pr = [&](auto get) { return make_float2(get(c), two ? get(c + 1) : 0.0f); };
          float2 lo = pr([&](int cc) { return Fx[cc * G::NFX + fx]; });
          float2 hi = pr([&](int cc) { return Fx[cc * G::NFX + fx + 1]; });
          float2 rhs = __fmul2_rn(__ffma2_rn(m1, lo, hi), c2(inv_h[0]));
          if constexpr (plane_dims(DIM) == 2) {
            lo = pr([&](int cc) { return Fy[cc * G::NFY + fy]; });
            hi = pr([&](int cc) { return Fy[cc * G::NFY + fy + BX]; });
            rhs = __ffma2_rn(__ffma2_rn(m1, lo, hi), c2(inv_h[1]), rhs);
          }
          if constexpr (ZS) {  // faces k + 1/2 and k - 1/2
            lo = pr([&](int cc) { return zf(k + 1, cc); });
            hi = pr([&](int cc) { return zf(k, cc); });
            rhs = __ffma2_rn(__ffma2_rn(m1, lo, hi), c2(inv_h[2]), rhs);
          }
          float2 o = rhs;
          if (!A.rhs_only) {
            o = __fmul2_rn(c2(A.b), __ffma2_rn(c2(dt), rhs, pr([&](int cc) { return us[cc]; })));
            if (A.Un) o = __ffma2_rn(c2(A.a), pr([&](int cc) { return un[cc]; }), o);
          }
          if (JF_CHECK(qc >= 0 && qc < A.N, "JFDBG store qc=%lld N=%lld\n", qc, A.N)) {
            A.out[qc + gcomp(DIM, c) * A.N] = o.x;
            if (two) A.out[qc + gcomp(DIM, c + 1) * A.N] = o.y;
          }
        };
        comb(0, true);
        comb(2, true);
        comb(4, false);
      }
    } else if (own) {
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        const int fx = ty * (BX + 1) + tx;
        T rhs = (Fx[c * G::NFX + fx + 1] - Fx[c * G::NFX + fx]) * inv_h[0];
        if (plane_dims(DIM) == 2) {
          const int fy = ty * BX + tx;
          rhs += (Fy[c * G::NFY + fy + BX] - Fy[c * G::NFY + fy]) * inv_h[1];
        }
        if constexpr (ZS) rhs += (zf(k, c) - zf(k + 1, c)) * inv_h[2];  // faces k + 1/2 and k - 1/2
        else if (marches(DIM)) rhs += (NFz_hi[c] - NFz_lo[c]) * inv_h[2];
        T o;
        if (A.rhs_only) {
          o = rhs;
        } else {
          o = A.b * (us[c] + dt * rhs);
          if (A.Un) o += A.a * un[c];
        }
        if (JF_CHECK(qc >= 0 && qc < A.N, "JFDBG store qc=%lld N=%lld\n", qc, A.N)) A.out[qc + gcomp(DIM, c) * A.N] = o;
      }
    }
    if (marches(DIM)) {
#pragma unroll
      for (int c = 0; c < 5; ++c) NFz_lo[c] = NFz_hi[c];  // (other schemes)
      const int nb = base + 1 == 6 ? 0 : base + 1;  // slot of plane k - 2, dead after this plane's faces
      if (k + 1 < z1) {
        commit_plane<T, BX, BY, DIM, VISC>(A, g, next, ring + nb * G::PLANE);  // plane k + 4
        if (!PC && k + 2 < z1) fetch_plane<T, BX, BY, DIM, VISC, WALLS>(A, next, gx0, gy0, k + 5);
      }
      __syncthreads();
      base = nb;
    }
  }
}

// ---------------------------------------------------------------------------
// Batched form: many independent grids (Section 4.5, feed_forward over a
// batch; sizes may differ), one persistent launch per RK stage.
template <typename T>
struct SimDesc {
  T* U;               // the simulation's field (caller-owned), [5][nz][ny][nx]
  T* U1;              // stage buffers (library-owned)
  T* U2;
  const double* dt;   // this simulation's step
  int nx, ny, nz;
  int periodic[3];
  int wall[3];
  T inv_h[3];
  long long N;
#ifdef JF_DEBUG_BOUNDS
  unsigned long long* trace;  // host-mapped trace records (debug build)
#endif
};

struct WorkItem {
  int sim;
  int bx, by;  // tile column (DIM_Y2: by = 0)
  int bz;      // z-march kernels (3D, DIM_Y2): the chunk of A0.zchunk planes (rows); else 0
};

// Arguments of batch stage `stage` for the simulation of descriptor d:
//   1: U1 = U + dt L(U) (every integrator); 2 (TVD-RK3): U2 = 3/4 U + 1/4 (U1 + dt L(U1));
//   3 (TVD-RK3): U = 1/3 U + 2/3 (U2 + dt L(U2)); 4 (TVD-RK2): U = 1/2 U + 1/2 (U1 + dt L(U1)).
// flag and (debug) trace are left as they are.
template <typename T>
__host__ __device__ __forceinline__ void batch_stage_args(const SimDesc<T>& d, int stage, StageArgs<T>& A) {
  A.nx = d.nx;
  A.ny = d.ny;
  A.nz = d.nz;
  A.N = d.N;
  for (int a = 0; a < 3; ++a) {
    A.periodic[a] = d.periodic[a];
    A.wall[a] = d.wall[a];
    A.inv_h[a] = d.inv_h[a];
  }
  A.dt = d.dt;
  A.rhs_only = 0;
  A.zchunk = d.nz;
  if (stage == 1) {
    A.Us = d.U; A.Un = nullptr; A.out = d.U1; A.a = T(0); A.b = T(1);
  } else if (stage == 2) {
    A.Us = d.U1; A.Un = d.U; A.out = d.U2; A.a = T(0.75); A.b = T(0.25);
  } else if (stage == 3) {
    A.Us = d.U2; A.Un = d.U; A.out = d.U; A.a = T(1.0 / 3.0); A.b = T(2.0 / 3.0);
  } else {
    A.Us = d.U1; A.Un = d.U; A.out = d.U; A.a = T(0.5); A.b = T(0.5);
  }
}

// DIM_Y2 launches: a 2D grid's arguments in the kernel's frame, its rows as
// the planes of the march (ny' = 1, nz' = ny; the y boundary condition and
// spacing move to the third axis; the kernel's y axis is inactive).
template <typename T>
__host__ __device__ __forceinline__ void rows_as_planes(StageArgs<T>& A) {
  A.nz = A.ny;
  A.ny = 1;
  A.periodic[2] = A.periodic[1];
  A.wall[2] = A.wall[1];
  A.inv_h[2] = A.inv_h[1];
  A.periodic[1] = 0;
  A.wall[1] = 0;
}

// Shared-memory elements of a tile: the plane ring and the face buffers.
template <typename T, int DIM, bool VISC, int BX, int BY>
constexpr size_t stage_smem_elems() {
  using G = Geo<BX, BY, DIM, VISC>;
  return (size_t)(G::RING * G::PLANE + 5 * G::NFX + 5 * G::NFY);
}

// Default scheme: the per-cell WENO5 face values of a plane, after the face
// buffers: x [2][5][BY][BX+2] (cells -1 .. BX of each row), y [2][5][BY+2][BX]
// (rows -1 .. BY); index 0 the value at the cell's right face, 1 at its left.
// 3D: then the z-face net fluxes [2][5][NCELL] and the upper WENO5 values of
// the columns' current cells [5][NCELL].
template <int DIM, int BX, int BY>
constexpr size_t recon_smem_elems() {
  return (size_t)2 * 5 * (BY * (BX + 2) + (plane_dims(DIM) == 2 ? (BY + 2) * BX : 0)) +
         (marches(DIM) ? 3 * 5 * BX * BY : 0);
}

// Element offset of the Rusanov-NN parameters in the dynamic shared memory:
// after the tile buffers, rounded up to 16 bytes (nn_alpha reads its weight
// rows with 16-byte loads).
template <typename T, int DIM, bool VISC, int BX, int BY>
constexpr size_t nn_smem_offset() {
  constexpr size_t q = 16 / sizeof(T);
  return (stage_smem_elems<T, DIM, VISC, BX, BY>() + q - 1) / q * q;
}

// The stage kernel.  blockDim.x == Geo::NT.
//  * Single grid (work == null): one CTA per tile, the tile from blockIdx;
//    grid = (ceil(nx/BX), ceil(ny/BY), ceil(nz/zchunk)) (3D), (.., .., 1) otherwise.
//  * Batch (work != null): persistent CTAs loop over the (simulation, tile)
//    work list in a static round robin (every item is one full tile of
//    equal cost); the grid arguments come from the simulation's descriptor,
//    stage 1: U1 = U + dt L(U); stage 2: U2 = 3/4 U + 1/4 (U1 + dt L(U1));
//    stage 3: U = 1/3 U + 2/3 (U2 + dt L(U2)); stage 4 (TVD-RK2):
//    U = 1/2 U + 1/2 (U1 + dt L(U1)).  z-march kernels (3D, DIM_Y2): an
//    item is a tile column and a chunk of A0.zchunk planes (rows).
// Both forms reach the tile computation through the same call below, so a
// simulation advanced in a batch is bitwise the one advanced alone.
template <typename T, int DIM, bool VISC, int BX, int BY, int MINB, int SCH>
__global__ void __launch_bounds__(Geo<BX, BY, DIM, VISC>::NT, MINB)
    stage_kernel(const StageArgs<T> A0, const SimDesc<T>* __restrict__ sims, const WorkItem* __restrict__ work,
                 int nwork, int stage, const Gas<T> g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
#ifdef JF_DEBUG_BOUNDS
  {
    unsigned dyn;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dyn));
    const size_t need = sizeof(T) * (SCH == SCH_NN ? nn_smem_offset<T, DIM, VISC, BX, BY>() + NN_PARAMS
                                                   : stage_smem_elems<T, DIM, VISC, BX, BY>() +
                                                         (sch_pc(SCH) ? recon_smem_elems<DIM, BX, BY>() : 0));
    if (!JF_CHECK(dyn >= need, "JFDBG smem %u < %llu\n", dyn, (unsigned long long)need)) return;
    if (work && threadIdx.x == 0)
      for (int i = blockIdx.x; i < nwork; i += gridDim.x) {
        const WorkItem w = work[i];
        const SimDesc<T> d = sims[w.sim];
        JF_CHECK(w.bx >= 0 && w.bx * BX < d.nx && w.by >= 0 && w.by * BY < d.ny,
                 "JFDBG work item %d sim %d tile (%d,%d) grid %dx%d\n", i, w.sim, w.bx, w.by, d.nx, d.ny);
      }
  }
  if (threadIdx.x == 0)
    jf_trace(A0.trace, 0x50, blockIdx.x, (unsigned long long)nwork, (unsigned long long)sims,
             (unsigned long long)work, (unsigned long long)stage, (unsigned long long)g.nn, 0);
#endif
  Gas<T> gk = g;
  if constexpr (SCH == SCH_NN) {
    // the Rusanov-NN parameters, after the stage buffers at a 16-byte
    // aligned offset (the launch adds them to the dynamic shared memory)
    T* th = reinterpret_cast<T*>(smem_raw) + nn_smem_offset<T, DIM, VISC, BX, BY>();
    for (int i = threadIdx.x; i < NN_PARAMS; i += blockDim.x) th[i] = __ldg(g.nn + i);
    __syncthreads();
    gk.nn = th;
  }
  for (int item = blockIdx.x;; item += gridDim.x) {
    StageArgs<T> A = A0;
    int bx = blockIdx.x, by = blockIdx.y, bz = blockIdx.z;
    if (work) {
      if (item >= nwork) break;
      const WorkItem w = work[item];
      const SimDesc<T> d = sims[w.sim];
      batch_stage_args(d, stage, A);
      if constexpr (DIM == DIM_Y2) rows_as_planes(A);
      if constexpr (marches(DIM)) A.zchunk = A0.zchunk;
      bx = w.bx;
      by = w.by;
      bz = w.bz;
#ifdef JF_DEBUG_BOUNDS
      if (threadIdx.x == 0)
        jf_trace(d.trace, 0x100 + stage, ((unsigned long long)item << 32) | (unsigned)w.sim,
                 ((unsigned long long)(unsigned)w.bx << 32) | (unsigned)w.by, (unsigned long long)A.Us,
                 (unsigned long long)A.out, (unsigned long long)A.Un, (unsigned long long)A.dt,
                 ((unsigned long long)(unsigned)A.nx << 32) | (unsigned)A.ny);
#endif
    } else if (item != (int)blockIdx.x) {
      break;
    }
    stage_tile<T, DIM, VISC, BX, BY, SCH>(A, gk, bx, by, bz, reinterpret_cast<T*>(smem_raw));
#ifdef JF_DEBUG_BOUNDS
    if (work && threadIdx.x == 0) jf_trace(sims[work[item].sim].trace, 0x200 + stage, item, 0, 0, 0, 0, 0, 0);
#endif
  }
}

template <typename T, int DIM, bool VISC, int BX, int BY>
constexpr size_t stage_smem_bytes() {
  return sizeof(T) * stage_smem_elems<T, DIM, VISC, BX, BY>();
}

}  // namespace jf

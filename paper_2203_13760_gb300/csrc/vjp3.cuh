// Adjoint of one Shu-Osher stage on 3D grids, marching along z (Sections
// 3.1-3.4, Section 7.2).  Same product as vjp_stage_kernel,
//   out = a1 x1 + a2 x2 + m + dt J(Us)^T m,   m = s_in lam,
// organised like the forward stage kernel instead of in boxes:
//
//  * A CTA owns a BX x BY column of cells and a chunk of planes along z.  It
//    evaluates every face it owns exactly once: the lower face of each of its
//    cells along x, y and z, and on a non-periodic axis also the upper
//    boundary face of the grid's last cell.  Every face of the grid is owned
//    by exactly one CTA, so no face is evaluated twice (the box kernel
//    evaluated the faces of a 5-cell halo around every box).
//  * The primitive variables (+T) of the planes k-3 .. k+2 live in a
//    six-slot shared-memory ring with a 3-cell x/y halo, and m = s_in lam of
//    the planes k-1, k in a two-slot ring with a 1-cell halo (zero on
//    zero-gradient ghosts: ghosts have no right-hand side).
//  * At face plane k the CTA runs the reverse passes of the x and y faces of
//    plane k and of the z face between planes k-1 and k (convective and, if
//    viscous, dissipative: the same per-face code as the box kernel).  Their
//    cotangents of W (+T) land on cells of the planes k-3 .. k+2 (tile plus a
//    3-cell halo) and are accumulated in a second six-slot shared-memory
//    ring with shared-memory atomics.
//  * Plane k-3 then receives nothing more from this CTA: its accumulator slot
//    is added to a global accumulator G[NCW][N] with global atomics, each
//    halo or ghost cell mapped to the cell it stands for (periodic wrap,
//    zero-gradient clamp: a ghost copies the boundary cell, so its cotangent
//    belongs to that cell), and the slot takes plane k+3.
//  * A per-cell pass (vjp3_finish_kernel) applies the transposed Jacobian of
//    W(U) and T = p / (rho R) to G and forms the stage combination.
//
// Summation order of the atomics, and so the last bits, may vary between
// runs, as in the box kernel.
#pragma once
#include "vjp.cuh"

namespace jf {

template <int BX, int BY, bool VISC>
struct V3Geo {
  static constexpr int H = 3;                        // halo of the W and accumulator planes
  static constexpr int PX = BX + 2 * H, PY = BY + 2 * H, CS = PX * PY;
  static constexpr int NCW = VISC ? 6 : 5;           // rho, u, v, w, p (, T)
  static constexpr int PLANE = NCW * CS;
  static constexpr int RING = 6;                     // planes k-3 .. k+2
  static constexpr int MPX = BX + 2, MPY = BY + 2, MCS = MPX * MPY;  // m planes, 1-cell halo
  // viscous: cotangents of the cell-centre tangential derivatives (the DC4
  // stencil is separable from the face's RC4): the x and y faces of the face
  // plane in 7 slots (spread along y: u, v; along x: u, v; along z: u, v, w),
  // the z faces in a ring of 4 planes (k-2 .. k+1) of 4 slots (spread along
  // x: w, u; along y: w, v)
  static constexpr int NXY = VISC ? 7 : 0, NZ = VISC ? 4 : 0, ZRING = 4;
};

template <typename T, bool VISC, int BX, int BY>
constexpr size_t vjp3_smem_bytes() {
  using G = V3Geo<BX, BY, VISC>;
  return sizeof(T) * (size_t)(2 * G::RING * G::PLANE + 2 * 5 * G::MCS + (G::NXY + G::ZRING * G::NZ) * G::CS);
}

// Accessor of the rings at face plane k: coordinates relative to the tile
// origin along x, y and to plane k along z (z in -3 .. 2 for W and the
// accumulator, -1 .. 0 for m).
template <typename T, bool VISC, int BX, int BY>
struct V3Tile {
  using G = V3Geo<BX, BY, VISC>;
  static constexpr int NCB = 0;
  static constexpr bool SEP3 = VISC;  // tangential cotangents through add_sep
  const T* W;
  T* acc;
  const T* M;
  T* cbxy;    // [7][PY][PX]
  T* cbz;     // [4 planes][4][PY][PX]
  int wp[6];  // element offset of the W / accumulator slot of plane k + z, index z + 3
  int mp[2];  // element offset of the m slot of plane k + z, index z + 1
  int zp[4];  // element offset of the z-face cotangent slot of plane k + z, index z + 2
  __device__ __forceinline__ T w(int c, int x, int y, int z) const {
    return W[wp[z + 3] + c * G::CS + (y + G::H) * G::PX + x + G::H];
  }
  __device__ __forceinline__ void add(int c, int x, int y, int z, T v) const {
    atomicAdd(acc + wp[z + 3] + c * G::CS + (y + G::H) * G::PX + x + G::H, v);
  }
  __device__ __forceinline__ T m(int c, int x, int y, int z) const {
    return M[mp[z + 1] + c * G::MCS + (y + 1) * G::MPX + x + 1];
  }
  // cotangent of the centre derivative of component c along axis e at a
  // cell of a face normal to d (x, y faces: plane k; z faces: planes k-2 .. k+1)
  __device__ __forceinline__ void add_sep(int d, int e, int c, int x, int y, int z, T v) const {
    const int cell = (y + G::H) * G::PX + x + G::H;
    if (d == 2) {
      const int slot = e == 0 ? (c == 3 ? 0 : 1) : (c == 3 ? 2 : 3);
      atomicAdd(cbz + zp[z + 2] + slot * G::CS + cell, v);
    } else {
      const int slot = e == 1 ? (c == 1 ? 0 : 1) : (e == 0 ? (c == 1 ? 2 : 3) : (c == 1 ? 4 : (c == 2 ? 5 : 6)));
      atomicAdd(cbxy + slot * G::CS + cell, v);
    }
  }
};

// Transposed DC4 along x or y at plane cell t of a cotangent slot src: the
// sum over o of dcw[o] src(t - dco[o] e) (dco = -2, -1, 1, 2; dcw = (1, -8, 8,
// -1) / 12); cells beyond the plane region hold no cotangent.
template <typename T, int BX, int BY, bool VISC>
__device__ __forceinline__ T vjp3_pull(const T* src, int t, int axis) {
  using G = V3Geo<BX, BY, VISC>;
  const int ly = t / G::PX, lx = t - ly * G::PX;
  const int pos = axis == 0 ? lx : ly, len = axis == 0 ? G::PX : G::PY, step = axis == 0 ? 1 : G::PX;
  T v = T(0);
  if (pos + 2 < len) v += (T(1) / T(12)) * src[t + 2 * step];
  if (pos + 1 < len) v += (-T(8) / T(12)) * src[t + step];
  if (pos >= 1) v += (T(8) / T(12)) * src[t - step];
  if (pos >= 2) v += (-T(1) / T(12)) * src[t - 2 * step];
  return v;
}

// Primitives (+T) of plane gz (unmapped) into W slot dst.
template <typename T, bool VISC, int BX, int BY, int NT>
__device__ __forceinline__ void vjp3_load_w(const VjpArgs<T>& A, const Gas<T>& g, T* dst, int x0, int y0, int gz,
                                            bool& bad) {
  using G = V3Geo<BX, BY, VISC>;
  const int kz = map_index(gz, A.n[2], A.periodic[2]);
  for (int t = threadIdx.x; t < G::CS; t += NT) {
    const int ly = t / G::PX, lx = t - ly * G::PX;
    const int gx = map_index(x0 + lx - G::H, A.n[0], A.periodic[0]);
    const int gy = map_index(y0 + ly - G::H, A.n[1], A.periodic[1]);
    const long long q = ((long long)kz * A.n[1] + gy) * A.n[0] + gx;
    const T r = A.Us[q];
    const T inv = trcp(r);
    const T u = A.Us[q + A.N] * inv, v = A.Us[q + 2 * A.N] * inv, w = A.Us[q + 3 * A.N] * inv;
    const T p = g.gm1 * (A.Us[q + 4 * A.N] - T(0.5) * r * (u * u + v * v + w * w));
    bad |= !(r > T(0)) || !(p > T(0));
    dst[t] = r;
    dst[G::CS + t] = u;
    dst[2 * G::CS + t] = v;
    dst[3 * G::CS + t] = w;
    dst[4 * G::CS + t] = p;
    if (VISC) dst[5 * G::CS + t] = p * inv * g.inv_R;
  }
}

// m = s_in lam of plane gz (unmapped) into m slot dst; zero on zero-gradient ghosts.
template <typename T, bool VISC, int BX, int BY, int NT>
__device__ __forceinline__ void vjp3_load_m(const VjpArgs<T>& A, T* dst, int x0, int y0, int gz) {
  using G = V3Geo<BX, BY, VISC>;
  const bool gzout = !A.periodic[2] && (gz < 0 || gz >= A.n[2]);
  const int kz = map_index(gz, A.n[2], A.periodic[2]);
  for (int t = threadIdx.x; t < G::MCS; t += NT) {
    const int ly = t / G::MPX, lx = t - ly * G::MPX;
    const int rx = x0 + lx - 1, ry = y0 + ly - 1;
    const bool ghost = gzout || (!A.periodic[0] && (rx < 0 || rx >= A.n[0])) ||
                       (!A.periodic[1] && (ry < 0 || ry >= A.n[1]));
    const int gx = map_index(rx, A.n[0], A.periodic[0]);
    const int gy = map_index(ry, A.n[1], A.periodic[1]);
    const long long q = ((long long)kz * A.n[1] + gy) * A.n[0] + gx;
#pragma unroll
    for (int c = 0; c < 5; ++c) dst[c * G::MCS + t] = ghost ? T(0) : A.s_in * A.lam[q + c * A.N];
  }
}

// The next W plane and m plane of the march in registers: their global loads
// are issued right after a face phase (vjp3_fetch), so that their latency
// overlaps with the gather passes and the accumulator flush, and converted
// and stored afterwards (vjp3_commit) -- the same values as vjp3_load_w and
// vjp3_load_m.
template <typename T, bool VISC, int BX, int BY, int NT>
struct V3Fetch {
  using G = V3Geo<BX, BY, VISC>;
  static constexpr int PW = (G::CS + NT - 1) / NT, PM = (G::MCS + NT - 1) / NT;
  T w[PW][5];
  T m[PM][5];
  bool ghost[PM];
};

template <typename T, bool VISC, int BX, int BY, int NT>
__device__ __forceinline__ void vjp3_fetch(const VjpArgs<T>& A, V3Fetch<T, VISC, BX, BY, NT>& f, int x0, int y0,
                                           int gzw, int gzm) {
  using G = V3Geo<BX, BY, VISC>;
  using F = V3Fetch<T, VISC, BX, BY, NT>;
  const int kw = map_index(gzw, A.n[2], A.periodic[2]);
#pragma unroll
  for (int i = 0; i < F::PW; ++i) {
    const int t = threadIdx.x + i * NT;
    if (t < G::CS) {
      const int ly = t / G::PX, lx = t - ly * G::PX;
      const int gx = map_index(x0 + lx - G::H, A.n[0], A.periodic[0]);
      const int gy = map_index(y0 + ly - G::H, A.n[1], A.periodic[1]);
      const long long q = ((long long)kw * A.n[1] + gy) * A.n[0] + gx;
#pragma unroll
      for (int c = 0; c < 5; ++c) f.w[i][c] = A.Us[q + c * A.N];
    }
  }
  const bool gzout = !A.periodic[2] && (gzm < 0 || gzm >= A.n[2]);
  const int km = map_index(gzm, A.n[2], A.periodic[2]);
#pragma unroll
  for (int i = 0; i < F::PM; ++i) {
    const int t = threadIdx.x + i * NT;
    if (t < G::MCS) {
      const int ly = t / G::MPX, lx = t - ly * G::MPX;
      const int rx = x0 + lx - 1, ry = y0 + ly - 1;
      f.ghost[i] = gzout || (!A.periodic[0] && (rx < 0 || rx >= A.n[0])) ||
                   (!A.periodic[1] && (ry < 0 || ry >= A.n[1]));
      const int gx = map_index(rx, A.n[0], A.periodic[0]);
      const int gy = map_index(ry, A.n[1], A.periodic[1]);
      const long long q = ((long long)km * A.n[1] + gy) * A.n[0] + gx;
#pragma unroll
      for (int c = 0; c < 5; ++c) f.m[i][c] = f.ghost[i] ? T(0) : A.lam[q + c * A.N];
    }
  }
}

template <typename T, bool VISC, int BX, int BY, int NT>
__device__ __forceinline__ void vjp3_commit(const VjpArgs<T>& A, const Gas<T>& g, const V3Fetch<T, VISC, BX, BY, NT>& f,
                                            T* dstw, T* dstm, bool& bad) {
  using G = V3Geo<BX, BY, VISC>;
  using F = V3Fetch<T, VISC, BX, BY, NT>;
#pragma unroll
  for (int i = 0; i < F::PW; ++i) {
    const int t = threadIdx.x + i * NT;
    if (t < G::CS) {
      const T r = f.w[i][0];
      const T inv = trcp(r);
      const T u = f.w[i][1] * inv, v = f.w[i][2] * inv, w = f.w[i][3] * inv;
      const T p = g.gm1 * (f.w[i][4] - T(0.5) * r * (u * u + v * v + w * w));
      bad |= !(r > T(0)) || !(p > T(0));
      dstw[t] = r;
      dstw[G::CS + t] = u;
      dstw[2 * G::CS + t] = v;
      dstw[3 * G::CS + t] = w;
      dstw[4 * G::CS + t] = p;
      if (VISC) dstw[5 * G::CS + t] = p * inv * g.inv_R;
    }
  }
#pragma unroll
  for (int i = 0; i < F::PM; ++i) {
    const int t = threadIdx.x + i * NT;
    if (t < G::MCS) {
#pragma unroll
      for (int c = 0; c < 5; ++c) dstm[c * G::MCS + t] = f.ghost[i] ? T(0) : A.s_in * f.m[i][c];
    }
  }
}

// Accumulator slot src (plane gz, unmapped) added to Gacc and cleared: a
// thread per plane cell maps the cell once and adds its components.
template <typename T, bool VISC, int BX, int BY, int NT>
__device__ __forceinline__ void vjp3_flush(const VjpArgs<T>& A, T* src, T* __restrict__ Gacc, int x0, int y0,
                                           int gz) {
  using G = V3Geo<BX, BY, VISC>;
  const int kz = map_index(gz, A.n[2], A.periodic[2]);
  for (int t = threadIdx.x; t < G::CS; t += NT) {
    const int ly = t / G::PX, lx = t - ly * G::PX;
    const int gx = map_index(x0 + lx - G::H, A.n[0], A.periodic[0]);
    const int gy = map_index(y0 + ly - G::H, A.n[1], A.periodic[1]);
    const long long q = ((long long)kz * A.n[1] + gy) * A.n[0] + gx;
#pragma unroll
    for (int c = 0; c < G::NCW; ++c) {
      const T v = src[c * G::CS + t];
      if (v != T(0)) {
        atomicAdd(Gacc + (long long)c * A.N + q, v);
        src[c * G::CS + t] = T(0);
      }
    }
  }
}

// The face reverse passes.  blockDim.x == NT; grid = (ceil(nx/BX),
// ceil(ny/BY), ceil(nz/zchunk)).  Gacc [NCW][N] must be zero on entry.
template <typename T, bool VISC, int BX, int BY, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB)
    vjp3_kernel(const VjpArgs<T> A, const Gas<T> g, T* __restrict__ Gacc, int zchunk) {
  using G = V3Geo<BX, BY, VISC>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Wr = reinterpret_cast<T*>(smem_raw);  // [RING][NCW][PY][PX]
  T* Ar = Wr + G::RING * G::PLANE;         // [RING][NCW][PY][PX]
  T* Mr = Ar + G::RING * G::PLANE;         // [2][5][MPY][MPX]
  T* Cxy = Mr + 2 * 5 * G::MCS;            // viscous: [7][PY][PX]
  T* Cz = Cxy + G::NXY * G::CS;            // viscous: [4 planes][4][PY][PX]
  const int nx = A.n[0], ny = A.n[1], nz = A.n[2];
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
  const int z0 = blockIdx.z * zchunk, z1 = min(z0 + zchunk, nz);
  const int ex = min(BX, nx - x0), ey = min(BY, ny - y0);
  // owned faces per row / column: the lower faces of the tile's cells, plus
  // the upper boundary face of the grid's last cell on a non-periodic axis
  const int fx = ex + ((!A.periodic[0] && x0 + BX >= nx) ? 1 : 0);
  const int fy = ey + ((!A.periodic[1] && y0 + BY >= ny) ? 1 : 0);
  const int kend = z1 + ((!A.periodic[2] && z1 == nz) ? 1 : 0);  // face plane nz: the top boundary z face
  // task decoding divides by fx and ex (1 .. BX + 1): for d >= 2,
  // r / d = (r m_d) >> 32 with m_d = ceil(2^32 / d) < 2^32, exact for
  // r < 2^16 (the error r (m_d - 2^32/d) / 2^32 < 2^-16 stays below 1/d);
  // d = 1 keeps r (m = 0 flags it)
  const unsigned mfx = fx > 1 ? 0xffffffffu / (unsigned)fx + 1u : 0u;
  const unsigned mex = ex > 1 ? 0xffffffffu / (unsigned)ex + 1u : 0u;
  auto divu = [](int r, unsigned m) { return m ? (int)__umulhi((unsigned)r, m) : r; };
  const T inv_h[3] = {A.inv_h[0], A.inv_h[1], A.inv_h[2]};

  bool bad = false;
  for (int q = 0; q < G::RING; ++q)
    vjp3_load_w<T, VISC, BX, BY, NT>(A, g, Wr + q * G::PLANE, x0, y0, z0 - 3 + q, bad);
  for (int t = threadIdx.x; t < G::RING * G::PLANE; t += NT) Ar[t] = T(0);
  for (int t = threadIdx.x; t < (G::NXY + G::ZRING * G::NZ) * G::CS; t += NT) Cxy[t] = T(0);
  vjp3_load_m<T, VISC, BX, BY, NT>(A, Mr, x0, y0, z0 - 1);
  vjp3_load_m<T, VISC, BX, BY, NT>(A, Mr + 5 * G::MCS, x0, y0, z0);
  if (bad) atomicOr(A.flag, 1);
  __syncthreads();

  V3Tile<T, VISC, BX, BY> V;
  V.W = Wr;
  V.acc = Ar;
  V.M = Mr;
  V.cbxy = Cxy;
  V.cbz = Cz;
  // the z-face cotangents of plane p sit in ring slot (p - z0 + 2) mod 4
  auto zslot = [&](int p) { return ((p - z0 + 2) & 3) * G::NZ * G::CS; };
  // transposed DC4 along x and y of the z-face cotangents of plane p into
  // its accumulator slot (thread per plane cell; no other thread writes the
  // cell meanwhile)
  auto gather_z = [&](int p) {
    if constexpr (VISC) {
      const T* src = Cz + zslot(p);
      T* dst = Ar + ((p - z0 + 3) % G::RING) * G::PLANE;
      for (int t = threadIdx.x; t < G::CS; t += NT) {
        dst[3 * G::CS + t] += vjp3_pull<T, BX, BY, VISC>(src, t, 0) + vjp3_pull<T, BX, BY, VISC>(src + 2 * G::CS, t, 1);
        dst[G::CS + t] += vjp3_pull<T, BX, BY, VISC>(src + G::CS, t, 0);
        dst[2 * G::CS + t] += vjp3_pull<T, BX, BY, VISC>(src + 3 * G::CS, t, 1);
      }
    }
  };
  for (int k = z0; k < kend; ++k) {
    const int b = (k - z0) % G::RING;  // slot of plane k - 3
#pragma unroll
    for (int z = -3; z <= 2; ++z) {
      int s = b + z + 3;
      s = s >= G::RING ? s - G::RING : s;
      V.wp[z + 3] = s * G::PLANE;
    }
    V.mp[0] = ((k - z0) & 1) * 5 * G::MCS;
    V.mp[1] = ((k - z0 + 1) & 1) * 5 * G::MCS;
#pragma unroll
    for (int z = -2; z <= 1; ++z) V.zp[z + 2] = zslot(k + z);

    auto face_nu = [&](auto dtag, const int p[3], T nu[5]) -> bool {
      constexpr int d = decltype(dtag)::value;
      const T h = inv_h[d];
      bool any = false;
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        nu[c] = (V.m(c, p[0], p[1], p[2]) - V.m(c, p[0] + (d == 0), p[1] + (d == 1), p[2] + (d == 2))) * h;
        any |= nu[c] != T(0);
      }
      return any;
    };
    auto run_face = [&](auto dtag, const int p[3], bool visc) {
      constexpr int d = decltype(dtag)::value;
      const Frame F{d, (d + 1) % 3, (d + 2) % 3};
      T nu[5];
      if (!face_nu(dtag, p, nu)) return;
      if (VISC && visc)
        visc_face_vjp<T, 3, VISC>(V, F, p, nu, g, inv_h);
      else
        conv_face_vjp<T, 3, VISC>(V, F, p, nu, g);
    };

    const bool xy = k < z1;  // plane nz (top boundary) has only its z face
    const int nfx = xy ? ey * fx : 0, nfy = xy ? fy * ex : 0, nfz = ex * ey;
    const int nconv = nfx + nfy + nfz;
    const int total = VISC ? 2 * nconv : nconv;
    for (int t = threadIdx.x; t < total; t += NT) {
      int r = t;
      const bool visc = VISC && r >= nconv;
      if (visc) r -= nconv;
      if (r < nfx) {  // x face: lower face of cell (x0 + f, y0 + j, k)
        const int j = divu(r, mfx), f = r - j * fx;
        const int p[3] = {f - 1, j, 0};
        run_face(std::integral_constant<int, 0>{}, p, visc);
      } else if ((r -= nfx) < nfy) {  // y face: lower face of cell (x0 + i, y0 + f, k)
        const int f = divu(r, mex), i = r - f * ex;
        const int p[3] = {i, f - 1, 0};
        run_face(std::integral_constant<int, 1>{}, p, visc);
      } else {  // z face between planes k - 1 and k
        r -= nfy;
        const int j = divu(r, mex), i = r - j * ex;
        const int p[3] = {i, j, -1};
        run_face(std::integral_constant<int, 2>{}, p, visc);
      }
    }
    __syncthreads();
    // W of plane k + 3 (slot b, last read by this face phase) and m of plane
    // k + 1 (the slot of plane k - 1) in flight during the passes below
    V3Fetch<T, VISC, BX, BY, NT> nxt;
    const bool more = k + 1 < kend;
    if (more) vjp3_fetch<T, VISC, BX, BY, NT>(A, nxt, x0, y0, k + 3, k + 1);
    if constexpr (VISC) {
      // the x and y faces' centre-derivative cotangents of plane k: transposed
      // DC4 along y and x into plane k, along z into planes k -+ 1, 2; the
      // z faces' of plane k - 2 are complete (their faces lie at planes up to
      // k - 1 / k): along x and y into plane k - 2
      constexpr int dco[4] = {-2, -1, 1, 2};
      constexpr T dcw[4] = {T(1) / T(12), -T(8) / T(12), T(8) / T(12), -T(1) / T(12)};
      T* a0 = Ar + V.wp[3];
      for (int t = threadIdx.x; t < G::CS; t += NT) {
        a0[G::CS + t] += vjp3_pull<T, BX, BY, VISC>(Cxy, t, 1) + vjp3_pull<T, BX, BY, VISC>(Cxy + 2 * G::CS, t, 0);
        a0[2 * G::CS + t] +=
            vjp3_pull<T, BX, BY, VISC>(Cxy + G::CS, t, 1) + vjp3_pull<T, BX, BY, VISC>(Cxy + 3 * G::CS, t, 0);
        const T zu = Cxy[4 * G::CS + t], zv = Cxy[5 * G::CS + t], zw = Cxy[6 * G::CS + t];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
          T* ao = Ar + V.wp[dco[o] + 3];
          ao[G::CS + t] += dcw[o] * zu;
          ao[2 * G::CS + t] += dcw[o] * zv;
          ao[3 * G::CS + t] += dcw[o] * zw;
        }
      }
      gather_z(k - 2);
      __syncthreads();
      for (int t = threadIdx.x; t < G::NXY * G::CS; t += NT) Cxy[t] = T(0);
      T* cz = Cz + zslot(k - 2);  // becomes plane k + 2
      for (int t = threadIdx.x; t < G::NZ * G::CS; t += NT) cz[t] = T(0);
    }
    // plane k - 3 is complete: add it to the global accumulator, then its
    // slots take plane k + 3 (W, cleared accumulator) and the m slot of plane
    // k - 1 takes plane k + 1
    vjp3_flush<T, VISC, BX, BY, NT>(A, Ar + b * G::PLANE, Gacc, x0, y0, k - 3);
    if (more) vjp3_commit<T, VISC, BX, BY, NT>(A, g, nxt, Wr + b * G::PLANE, Mr + ((k - z0) & 1) * 5 * G::MCS, bad);
    __syncthreads();
  }
  // the z-face cotangents still held (planes kend - 2 .. kend), then the
  // planes still held: kend - 3 .. kend + 1
  if constexpr (VISC) {
    for (int pl = kend - 2; pl <= kend; ++pl) gather_z(pl);
    __syncthreads();
  }
  for (int pl = kend - 3; pl <= kend + 1; ++pl) {
    int s = (pl - z0 + 3) % G::RING;
    vjp3_flush<T, VISC, BX, BY, NT>(A, Ar + s * G::PLANE, Gacc, x0, y0, pl);
  }
  if (bad) atomicOr(A.flag, 1);
}

// Per cell: cotangent of W (+T) in Gacc -> cotangent of U (transposed
// Jacobian of W(U), and of T = p / (rho R)), then
// out = m + dt J^T m + a1 x1 + a2 x2.
template <typename T, bool VISC>
__global__ void __launch_bounds__(256) vjp3_finish_kernel(const VjpArgs<T> A, const Gas<T> g,
                                                          const T* __restrict__ Gacc) {
  const long long N = A.N;
  const T dt = T(*A.dt);
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += (long long)gridDim.x * blockDim.x) {
    const T r = A.Us[q];
    const T inv = trcp(r);
    const T u = A.Us[q + N] * inv, v = A.Us[q + 2 * N] * inv, w = A.Us[q + 3 * N] * inv;
    const T p = g.gm1 * (A.Us[q + 4 * N] - T(0.5) * r * (u * u + v * v + w * w));
    T br = Gacc[q], bu = Gacc[q + N], bv = Gacc[q + 2 * N], bw = Gacc[q + 3 * N], bp = Gacc[q + 4 * N];
    if (VISC) {
      const T bT = Gacc[q + 5 * N];
      const T Tc = p * inv * g.inv_R;
      br -= bT * Tc * inv;  // T = p / (rho R)
      bp += bT * Tc * trcp(p);
    }
    T bU[5];
    bU[0] = br - (bu * u + bv * v + bw * w) * inv + bp * g.gm1 * T(0.5) * (u * u + v * v + w * w);
    bU[1] = bu * inv - bp * g.gm1 * u;
    bU[2] = bv * inv - bp * g.gm1 * v;
    bU[3] = bw * inv - bp * g.gm1 * w;
    bU[4] = bp * g.gm1;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
      T o = A.s_in * A.lam[q + c * N] + dt * bU[c];
      if (A.x1) o += A.a1 * A.x1[q + c * N];
      if (A.x2) o += A.a2 * A.x2[q + c * N];
      A.out[q + c * N] = o;
    }
  }
}

}  // namespace jf

// FP64 reductions of libjf: the CFL time step (Section 3.2) and the density
// mismatch loss of the adjoint workload (Section 7.2, a squared-error state
// loss).
//
// Both are single launches: each CTA reduces its cells (warp shuffles, then
// shared memory) and folds its result into a global accumulator with one
// atomic; the last CTA to finish (ticket counter) finalises the result and
// resets the accumulator and counter for the next launch.  No CTA waits for
// another.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "jf_math.cuh"

namespace jf {

struct CflArgs {
  long long N;        // cells
  int nactive;        // active axes (velocity components that count), 1..3
  double gamma;
  double kdiff;       // max(mu, lambda / c_v) if dissipative, else 0
  double hmin;        // min_d dx_d over active axes
  double cfl;
};

// Scratch of the reductions (device memory owned by the caller).
struct ReduceScratch {
  unsigned long long acc[2];  // bit patterns of non-negative doubles (ordered like the values)
  unsigned int ticket;
  unsigned int pad;
  double sum;
};

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per-cell rates of the CFL criterion, folded into running maxima: the wave
// rate max_d |u_d| + c over the active axes and the diffusion rate kdiff / rho.
// Computed in the field's precision (FP64 units are scarce on this part); the
// maxima are later formed in FP64, and a rate converted to FP64 is exact, so
// the result is the exact maximum of the per-cell values.
template <typename T>
__device__ __forceinline__ void cell_rates_of(T r, T ru, T rv, T rw, T E, int nactive, T gamma, T gm1, T kdiff,
                                              T& conv, T& diff, bool& bad) {
  const T inv = T(1) / r;
  const T u = ru * inv;
  const T v = rv * inv;
  const T w = rw * inv;
  const T p = gm1 * (E - T(0.5) * r * (u * u + v * v + w * w));
  bad |= !(r > T(0)) || !(p > T(0));
  const T c = tsqrt(gamma * p * inv);
  T m = fabs(u);
  if (nactive > 1) m = fmax(m, fabs(v));
  if (nactive > 2) m = fmax(m, fabs(w));
  conv = fmax(conv, m + c);
  diff = fmax(diff, kdiff * inv);
}
template <typename T>
__device__ __forceinline__ void cell_rates(const T* __restrict__ U, long long q, long long N, int nactive, T gamma,
                                           T gm1, T kdiff, T& conv, T& diff, bool& bad) {
  cell_rates_of(U[q], U[q + N], U[q + 2 * N], U[q + 3 * N], U[q + 4 * N], nactive, gamma, gm1, kdiff, conv, diff,
                bad);
}

// 16-byte vectors of cells (4 in FP32, 2 in FP64) for the CFL pass
__device__ __forceinline__ void unpack(const float4& a, float o[4]) { o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; }
__device__ __forceinline__ void unpack(const double2& a, double o[2]) { o[0] = a.x; o[1] = a.y; }
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };

// Block-wide FP64 maxima of (conv, diff) folded into sc; the CTA that takes
// the last of `nblocks` tickets forms dt = CFL min(hmin / C, 3/14 hmin^2 / D)
// and resets sc.  blockDim.x <= 256, a multiple of 32.
__device__ __forceinline__ void finish_cfl(double conv, double diff, ReduceScratch* sc, unsigned int nblocks,
                                           double hmin, double cfl, double* dt_out, double* dt_out2) {
  __shared__ double s_conv[8], s_diff[8];
  conv = warp_max(conv);
  diff = warp_max(diff);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { s_conv[wid] = conv; s_diff[wid] = diff; }
  __syncthreads();
  if (wid == 0) {
    conv = lane < (int)(blockDim.x >> 5) ? s_conv[lane] : 0.0;
    diff = lane < (int)(blockDim.x >> 5) ? s_diff[lane] : 0.0;
    conv = warp_max(conv);
    diff = warp_max(diff);
    if (lane == 0) {
      // NaN never wins fmax; a NaN state is reported through the flag
      atomicMax(&sc->acc[0], (unsigned long long)__double_as_longlong(conv));
      atomicMax(&sc->acc[1], (unsigned long long)__double_as_longlong(diff));
      __threadfence();
      const unsigned int t = atomicAdd(&sc->ticket, 1u);
      if (t == nblocks - 1) {
        __threadfence();
        const double C = __longlong_as_double((long long)atomicMax(&sc->acc[0], 0ull));
        const double Dm = __longlong_as_double((long long)atomicMax(&sc->acc[1], 0ull));
        double dt = hmin / C;
        if (Dm > 0.0) dt = fmin(dt, (3.0 / 14.0) * hmin * hmin / Dm);
        dt *= cfl;
        *dt_out = dt;
        if (dt_out2) *dt_out2 = dt;
        sc->acc[0] = 0ull;
        sc->acc[1] = 0ull;
        sc->ticket = 0u;
        __threadfence();
      }
    }
  }
}

// loss = sum_cells (rho - target)^2 * dV; seed = d loss / dU (density
// component only).  blockDim.x == 256.
template <typename T>
__global__ void __launch_bounds__(256) loss_density_kernel(const T* __restrict__ U, const T* __restrict__ target,
                                                           long long N, double dV, ReduceScratch* sc,
                                                           double* loss, T* seed) {
  double s = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < N; q += stride) {
    const double d = (double)U[q] - (double)target[q];
    s += d * d * dV;
    if (seed) {
      seed[q] = (T)(2.0 * d * dV);
      seed[q + N] = T(0);
      seed[q + 2 * N] = T(0);
      seed[q + 3 * N] = T(0);
      seed[q + 4 * N] = T(0);
    }
  }
  __shared__ double s_sum[8];
  s = warp_sum(s);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) s_sum[wid] = s;
  __syncthreads();
  if (wid == 0) {
    s = lane < (int)(blockDim.x >> 5) ? s_sum[lane] : 0.0;
    s = warp_sum(s);
    if (lane == 0) {
      atomicAdd(&sc->sum, s);
      __threadfence();
      const unsigned int t = atomicAdd(&sc->ticket, 1u);
      if (t == gridDim.x - 1) {
        __threadfence();
        *loss = atomicAdd(&sc->sum, 0.0);
        sc->sum = 0.0;
        sc->ticket = 0u;
        __threadfence();
      }
    }
  }
}

// Section 7.4 training loss: the mean square difference of the primitive
// state vectors of nstates states U and Uref (each [5][ncells], stored one
// after another), over the states, the cells and ncomp components: (rho, u,
// v, p) for ncomp = 4 (two-dimensional states), (rho, u, v, w, p) for 5.
//   loss = 1/(nstates ncomp ncells) sum (W(U) - W(Uref))^2,
//   grad = d loss / dU: the cotangent g = 2 (W(U) - W(Uref)) / count of the
//   primitives through the transposed Jacobian of W(U) (u_i = m_i / rho,
//   p = (gamma - 1)(E - |m|^2 / (2 rho))).
// FP64 accumulation; the last CTA (ticket) writes the loss and resets sc.
template <typename T>
__global__ void __launch_bounds__(256) primitive_mse_kernel(const T* __restrict__ U, const T* __restrict__ Uref,
                                                            long long nstates, long long ncells, int ncomp,
                                                            double gm1, ReduceScratch* sc, double* loss, T* grad) {
  const long long total = nstates * ncells;
  const double inv_count = 1.0 / ((double)total * ncomp);
  double s = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += stride) {
    const long long st = q / ncells, i = q - st * ncells;
    const long long b = st * 5 * ncells + i;
    double W[5], D[5];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const T* X = side == 0 ? U : Uref;
      const double r = (double)X[b], ir = 1.0 / r;
      const double u = (double)X[b + ncells] * ir, v = (double)X[b + 2 * ncells] * ir;
      const double w = (double)X[b + 3 * ncells] * ir;
      const double p = gm1 * ((double)X[b + 4 * ncells] - 0.5 * r * (u * u + v * v + w * w));
      const double P[5] = {r, u, v, w, p};
#pragma unroll
      for (int c = 0; c < 5; ++c) {
        if (side == 0) W[c] = P[c];
        else D[c] = W[c] - P[c];
      }
    }
    if (ncomp == 4) D[3] = 0.0;
    s += D[0] * D[0] + D[1] * D[1] + D[2] * D[2] + D[3] * D[3] + D[4] * D[4];
    if (grad) {
      const double k = 2.0 * inv_count, ir = 1.0 / W[0];
      const double gr = k * D[0], gu = k * D[1], gv = k * D[2], gw = k * D[3], gp = k * D[4];
      grad[b] = (T)(gr - (gu * W[1] + gv * W[2] + gw * W[3]) * ir +
                    gp * gm1 * 0.5 * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]));
      grad[b + ncells] = (T)(gu * ir - gp * gm1 * W[1]);
      grad[b + 2 * ncells] = (T)(gv * ir - gp * gm1 * W[2]);
      grad[b + 3 * ncells] = (T)(gw * ir - gp * gm1 * W[3]);
      grad[b + 4 * ncells] = (T)(gp * gm1);
    }
  }
  __shared__ double s_sum[8];
  s = warp_sum(s);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) s_sum[wid] = s;
  __syncthreads();
  if (wid == 0) {
    s = lane < (int)(blockDim.x >> 5) ? s_sum[lane] : 0.0;
    s = warp_sum(s);
    if (lane == 0) {
      atomicAdd(&sc->sum, s);
      __threadfence();
      const unsigned int t = atomicAdd(&sc->ticket, 1u);
      if (t == gridDim.x - 1) {
        __threadfence();
        *loss = atomicAdd(&sc->sum, 0.0) * inv_count;
        sc->sum = 0.0;
        sc->ticket = 0u;
        __threadfence();
      }
    }
  }
}

}  // namespace jf

// The CFL reduction kernel (Section 3.2) for single grids and batches.
//
// Single grid (chunks == null): grid-stride over the cells of U, the last CTA
// (ticket) forms dt.  Batch (chunks != null): each CTA reduces one chunk of
// one simulation; the last chunk of a simulation forms that simulation's dt.
// Both forms run the same per-cell and reduction code, so a simulation's dt
// in a batch is bitwise the dt of the simulation run alone.
#pragma once
#include "reduce.cuh"
#include "stage.cuh"

namespace jf {

struct CflChunk {
  int sim;
  int nchunks;   // chunks of this simulation
  long long begin, end;
};

template <typename T>
__global__ void __launch_bounds__(256) cfl_kernel(const T* __restrict__ U0, CflArgs a0, ReduceScratch* sc0,
                                                  double* dt0, double* dt0b, int* flag,
                                                  const SimDesc<T>* __restrict__ sims,
                                                  const CflChunk* __restrict__ chunks,
                                                  const CflArgs* __restrict__ args, ReduceScratch* red,
                                                  double* dts) {
  const T* U;
  CflArgs a;
  ReduceScratch* sc;
  double *dto, *dto2;
  long long first, q0, end, stride;
  unsigned int nblocks;
  if (chunks) {
    const CflChunk ch = chunks[blockIdx.x];
    a = args[ch.sim];
    U = sims[ch.sim].U;
#ifdef JF_DEBUG_BOUNDS
    if (threadIdx.x == 0)
      jf_trace(sims[ch.sim].trace, 0x300, blockIdx.x, ch.sim, (unsigned long long)U, (unsigned long long)ch.begin,
               (unsigned long long)ch.end, (unsigned long long)a.N, (unsigned long long)(red + ch.sim));
#endif
    sc = red + ch.sim;
    dto = dts + ch.sim;
    dto2 = nullptr;
    first = ch.begin;
    q0 = ch.begin + threadIdx.x;
    end = ch.end;
    stride = blockDim.x;
    nblocks = (unsigned int)ch.nchunks;
  } else {
    a = a0;
    U = U0;
    sc = sc0;
    dto = dt0;
    dto2 = dt0b;
    first = 0;
    q0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    end = a.N;
    stride = (long long)gridDim.x * blockDim.x;
    nblocks = gridDim.x;
  }
  T conv = T(0), diff = T(0);
  const T gamma = (T)a.gamma, gm1 = (T)(a.gamma - 1.0), kdiff = (T)a.kdiff;
  bool bad = false;
  constexpr int V = 16 / (int)sizeof(T);  // cells per 16-byte vector
  if (a.N % V == 0 && first % V == 0 && end % V == 0) {
    // every component read in 16-byte vectors (U is 16-byte aligned, a
    // component spans a whole number of vectors, and so does a batch chunk);
    // the maxima are exact, so dt equals the scalar form's
    using VT = typename Vec16<T>::type;
    const VT* Uv = reinterpret_cast<const VT*>(U);
    const long long Nv = a.N / V;
    const long long vend = end / V;
    for (long long qv = first / V + (q0 - first); qv < vend; qv += stride) {
      T r[V], ru[V], rv[V], rw[V], E[V];
      unpack(Uv[qv], r);
      unpack(Uv[qv + Nv], ru);
      unpack(Uv[qv + 2 * Nv], rv);
      unpack(Uv[qv + 3 * Nv], rw);
      unpack(Uv[qv + 4 * Nv], E);
#pragma unroll
      for (int k = 0; k < V; ++k)
        cell_rates_of(r[k], ru[k], rv[k], rw[k], E[k], a.nactive, gamma, gm1, kdiff, conv, diff, bad);
    }
  } else {
    for (long long q = q0; q < end; q += stride) cell_rates(U, q, a.N, a.nactive, gamma, gm1, kdiff, conv, diff, bad);
  }
  if (bad) atomicOr(flag, 1);
  finish_cfl((double)conv, (double)diff, sc, nblocks, a.hmin, a.cfl, dto, dto2);
}

}  // namespace jf

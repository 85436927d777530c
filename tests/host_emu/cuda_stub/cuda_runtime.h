// Host stand-ins for the CUDA names that the stage kernel headers use, so
// that the kernel source compiles for the CPU in the host emulation test
// (tests/test_host_emulation.py): one std::thread per CUDA thread, a
// std::barrier per CTA, plain loads for __ldg, exact division for
// __fdividef, and per-lane fmaf / * / + for the packed FP32x2 operations.
#pragma once
#include <algorithm>
#include <barrier>
#include <cmath>
#include <cstdint>
#include <cstdio>
#define __host__
#define __device__
#define __global__
#define __forceinline__ inline
#define __noinline__ __attribute__((noinline))
#define __shared__
#define __launch_bounds__(...)
#define __align__(n) alignas(n)
#define __restrict__ __restrict
struct alignas(8) float2 { float x, y; };
struct alignas(16) double2 { double x, y; };
struct uint3 { unsigned x, y, z; };
struct dim3 { unsigned x = 1, y = 1, z = 1; };
typedef int cudaError_t;
typedef void* cudaStream_t;
inline float2 make_float2(float a, float b) { return float2{a, b}; }
extern thread_local uint3 threadIdx;
extern thread_local uint3 blockIdx;
extern dim3 blockDim, gridDim;
void emu_syncthreads();
#define __syncthreads() emu_syncthreads()
template <class T> inline T __ldg(const T* p) { return *p; }
inline float __fdividef(float a, float b) { return a / b; }
inline float2 __ffma2_rn(float2 a, float2 b, float2 c) { return float2{std::fmaf(a.x, b.x, c.x), std::fmaf(a.y, b.y, c.y)}; }
inline float2 __fmul2_rn(float2 a, float2 b) { return float2{a.x * b.x, a.y * b.y}; }
inline float2 __fadd2_rn(float2 a, float2 b) { return float2{a.x + b.x, a.y + b.y}; }
inline int atomicOr(int* p, int v) { return __atomic_fetch_or(p, v, __ATOMIC_RELAXED); }
inline int atomicAdd(int* p, int v) { return __atomic_fetch_add(p, v, __ATOMIC_RELAXED); }
inline unsigned long long atomicAdd(unsigned long long* p, unsigned long long v) {
  return __atomic_fetch_add(p, v, __ATOMIC_RELAXED);
}
inline void __threadfence_system() {}
using std::max;
using std::min;

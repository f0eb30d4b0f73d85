// Storage formats, per-size transform configurations, FP64 block sums and
// the "last block of a frame" pattern used for the CG scalars.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.cuh"

namespace sense {

// device error flag bits (plan workspace word, read by sense_plan_check)
constexpr int ERR_LINES = 1;    // a line index outside [0, ny) or not strictly increasing
constexpr int ERR_TIMEOUT = 2;  // a bounded wait gave up

// CG per-frame outcome codes (match sense_cg_outcome; 0 = still running)
constexpr int CG_RUNNING = 0, CG_CONVERGED = 1, CG_MAXITER = 2, CG_BREAKDOWN = 3;

// ---------------------------------------------------------------------------
// storage of S and y: complex64, or bfloat16 pairs (round-to-nearest-even on store)
// ---------------------------------------------------------------------------
struct StC64 {
  using T = float2;
  __device__ __forceinline__ static float2 ld(const T* p, size_t i) { return __ldg(p + i); }
  __device__ __forceinline__ static void st(T* p, size_t i, float2 v) { p[i] = v; }
};

struct StBF16 {
  using T = __nv_bfloat162;
  __device__ __forceinline__ static float2 ld(const T* p, size_t i) {
    unsigned u = __ldg(reinterpret_cast<const unsigned*>(p) + i);
    __nv_bfloat162 h;
    memcpy(&h, &u, 4);
    return __bfloat1622float2(h);
  }
  __device__ __forceinline__ static void st(T* p, size_t i, float2 v) { p[i] = __float22bfloat162_rn(v); }
};

// ---------------------------------------------------------------------------
// transform configuration per length: Col<N1, N2, T, W>
// (threads per block always a multiple of 32)
// ---------------------------------------------------------------------------
template <int N>
struct Cfg;
template <> struct Cfg<8> { using C = Col<4, 2, 2, 16>; };
template <> struct Cfg<12> { using C = Col<4, 3, 4, 16>; };
template <> struct Cfg<16> { using C = Col<4, 4, 4, 16>; };
template <> struct Cfg<20> { using C = Col<5, 4, 4, 16>; };
template <> struct Cfg<32> { using C = Col<8, 4, 4, 32>; };
template <> struct Cfg<64> { using C = Col<8, 8, 8, 32>; };
template <> struct Cfg<96> { using C = Col<12, 8, 8, 32>; };
template <> struct Cfg<128> { using C = Col<16, 8, 8, 32>; };
template <> struct Cfg<160> { using C = Col<10, 16, 16, 16>; };
template <> struct Cfg<192> { using C = Col<12, 16, 16, 16>; };
template <> struct Cfg<256> { using C = Col<16, 16, 16, 16>; };
template <> struct Cfg<320> { using C = Col<16, 20, 20, 16>; };
template <> struct Cfg<384> { using C = Col<16, 24, 24, 16>; };

#define SENSE_FOR_EACH_SIZE(X) \
  X(8) X(12) X(16) X(20) X(32) X(64) X(96) X(128) X(160) X(192) X(256) X(320) X(384)

// ---------------------------------------------------------------------------
// FP64 block sum; the result is valid in thread 0.  Fixed shuffle tree and a
// fixed warp order, so the value depends only on the inputs.
// ---------------------------------------------------------------------------
template <int THREADS>
__device__ __forceinline__ double block_sum(double v, double* red) {
  static_assert(THREADS % 32 == 0, "block size");
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
#pragma unroll 1
    for (int i = 0; i < THREADS / 32; ++i) s += red[i];
  }
  return s;
}

// Thread 0 publishes this block's partial, then counts arrivals for the
// frame; returns true (in thread 0 only) for the last block to arrive.  No
// block ever waits on another.
__device__ __forceinline__ bool publish_and_arrive(double partial, double* slot, unsigned* counter,
                                                   unsigned total) {
  bool last = false;
  if (threadIdx.x == 0) {
    *slot = partial;
    __threadfence();
    unsigned prev = atomicAdd(counter, 1u);
    last = (prev == total - 1);
    if (last) __threadfence();
  }
  return last;
}

// Ordered sum of `n` partials written by other blocks (bypasses L1).
__device__ __forceinline__ double ordered_sum(const double* part, int n) {
  double s = 0.0;
#pragma unroll 1
  for (int i = 0; i < n; ++i) s += __ldcg(part + i);
  return s;
}

// Per-frame CG state, device resident (plan workspace).
struct CgState {
  double* rho;     // <r, r>
  double* rho0;    // <r0, r0>
  double* alpha;
  double* beta;
  double* resid;   // sqrt(rho / rho0)
  int* iters;
  int* outcome;
  int* active;     // 1 while the frame iterates
  int* live;       // number of active frames (single counter)
  unsigned* counter;  // [F] arrival counters
  double* part;    // [F][part_stride] block partials
  int part_stride;
  double tol;
};

}  // namespace sense

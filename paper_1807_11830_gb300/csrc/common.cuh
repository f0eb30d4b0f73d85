// Storage formats, per-size transform configurations, FP64 block sums and
// the "last block of a frame" pattern used for the CG scalars.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "engine.cuh"
#include "tma.cuh"

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
  __device__ __forceinline__ static float2 lds(const T* p, int i) { return p[i]; }  // shared memory
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
  __device__ __forceinline__ static float2 lds(const T* p, int i) { return __bfloat1622float2(p[i]); }
  __device__ __forceinline__ static void st(T* p, size_t i, float2 v) { p[i] = __float22bfloat162_rn(v); }
};

// ---------------------------------------------------------------------------
// transform configuration per length: Col<T, W, Radices<...>>, each thread
// holding about 8 values per stage (threads per block a multiple of 32)
// ---------------------------------------------------------------------------
template <int N>
struct Cfg;
template <> struct Cfg<8> { using C = Col<2, 16, Radices<4, 2>>; };
template <> struct Cfg<12> { using C = Col<4, 16, Radices<4, 3>>; };
template <> struct Cfg<16> { using C = Col<4, 16, Radices<4, 4>>; };
template <> struct Cfg<20> { using C = Col<4, 16, Radices<5, 4>>; };
template <> struct Cfg<24> { using C = Col<4, 16, Radices<4, 6>>; };
template <> struct Cfg<32> { using C = Col<4, 32, Radices<8, 4>>; };
template <> struct Cfg<40> { using C = Col<8, 16, Radices<5, 8>>; };
template <> struct Cfg<48> { using C = Col<8, 16, Radices<6, 8>>; };
template <> struct Cfg<64> { using C = Col<8, 32, Radices<8, 8>>; };
template <> struct Cfg<80> { using C = Col<10, 16, Radices<8, 10>>; };
template <> struct Cfg<96> { using C = Col<24, 16, Radices<4, 4, 6>>; };
template <> struct Cfg<120> { using C = Col<12, 16, Radices<10, 12>>; };
template <> struct Cfg<128> { using C = Col<16, 16, Radices<8, 4, 4>>; };
template <> struct Cfg<144> { using C = Col<12, 16, Radices<12, 12>>; };
template <> struct Cfg<160> { using C = Col<20, 16, Radices<8, 4, 5>>; };
template <> struct Cfg<192> { using C = Col<24, 16, Radices<8, 3, 8>>; };
template <> struct Cfg<240> { using C = Col<16, 16, Radices<15, 16>>; };
template <> struct Cfg<256> { using C = Col<32, 16, Radices<8, 4, 8>>; };
template <> struct Cfg<288> { using C = Col<24, 16, Radices<6, 6, 8>>; };
template <> struct Cfg<320> { using C = Col<40, 16, Radices<8, 4, 10>>; };
template <> struct Cfg<384> { using C = Col<48, 16, Radices<8, 4, 12>>; };

// Variants of the normal-operator kernel per length: V = 0 is Cfg<N>; the
// others trade threads per column, tile width and a minimum number of
// resident blocks (which caps registers).  The autotuner times the variants
// that exist for a plan's length and keeps the fastest.
template <int N, int V>
struct NormCfg {
  static constexpr bool exists = (V == 0);
  using C = typename Cfg<N>::C;
  static constexpr int MINB = 1;
};
#define SENSE_NORM_VARIANT(N_, V_, MINB_, ...)   \
  template <>                                    \
  struct NormCfg<N_, V_> {                       \
    static constexpr bool exists = true;         \
    using C = __VA_ARGS__;                       \
    static constexpr int MINB = MINB_;           \
  };
SENSE_NORM_VARIANT(128, 1, 1, Col<8, 32, Radices<16, 8>>)
SENSE_NORM_VARIANT(128, 2, 4, WCol<16, 8, Radices<8, 4, 4>, Pads<Pad<4, 4>, Pad<1, 4>>>)
SENSE_NORM_VARIANT(192, 1, 1, Col<16, 16, Radices<12, 16>>)
SENSE_NORM_VARIANT(192, 2, 2, Col<24, 16, Radices<8, 3, 8>>)
SENSE_NORM_VARIANT(192, 3, 2, WCol<32, 8, Radices<8, 3, 8>, Pads<Pad<0, 2>, Pad<1, 4>>>)
SENSE_NORM_VARIANT(256, 1, 2, WCol<32, 8, Radices<8, 4, 8>, Pads<Pad<8, 5>, Pad<1, 4>>>)
SENSE_NORM_VARIANT(256, 2, 1, WCol<16, 8, Radices<16, 16>, Pads<Pad<1, 4>>>)
SENSE_NORM_VARIANT(256, 3, 2, Col<32, 8, Radices<8, 4, 8>>)
SENSE_NORM_VARIANT(320, 1, 1, Col<20, 16, Radices<16, 20>>)
SENSE_NORM_VARIANT(320, 2, 1, Col<40, 8, Radices<8, 4, 10>>)
SENSE_NORM_VARIANT(384, 1, 1, Col<24, 16, Radices<16, 24>>)
SENSE_NORM_VARIANT(384, 2, 1, Col<48, 8, Radices<8, 4, 12>>)
#undef SENSE_NORM_VARIANT
constexpr int kNormVariants = 4;

#define SENSE_FOR_EACH_SIZE(X)                                                                     \
  X(8) X(12) X(16) X(20) X(24) X(32) X(40) X(48) X(64) X(80) X(96) X(120) X(128) X(144) X(160) X(192) \
  X(240) X(256) X(288) X(320) X(384)

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

// Two-level mixed-radix transform of W independent length-N sequences held
// by one thread block ("columns" of a tile), N = N1 * N2.
//
// Thread layout: THREADS = T * W.  Thread (t, c) with c = tid % W the
// sequence (column) and t = tid / W its phase.  For W = 32 a warp is one t
// across 32 adjacent columns, so every global access of a warp is one
// contiguous 256-byte row segment and every shared access is one row.
//
// Index split (Cooley-Tukey, N = N1 N2):
//   sample n = N2*n1 + n2,   frequency k = k1 + N1*k2
//   X[k1 + N1 k2] = sum_n2 w_N2^{n2 k2} w_N^{n2 k1} sum_n1 x[N2 n1 + n2] w_N1^{n1 k1}
// Sample-side registers  xr[b][n1]: n2 = t + T*b  (B1 = ceil(N2/T) groups)
// Frequency-side registers kr[b][k2]: k1 = t + T*b (B2 = ceil(N1/T) groups)
// One shared-memory exchange moves data between the two layouts.  The
// exchange buffer holds element (k1, n2) of column c at
//   ((k1*N2 + n2) * W + c'),  c' = c, or c ^ 4 on odd (k1 + n2) when W = 8
// (the swizzle keeps half-warps conflict-free for 8-column tiles).
#pragma once
#include "codelets.cuh"

namespace sense {

template <int N1_, int N2_, int T_, int W_>
struct Col {
  static constexpr int N1 = N1_, N2 = N2_, T = T_, W = W_;
  static constexpr int N = N1 * N2;
  static constexpr int B1 = (N2 + T - 1) / T;
  static constexpr int B2 = (N1 + T - 1) / T;
  static constexpr int THREADS = T * W;
  static constexpr bool FULL1 = (B1 * T == N2);
  static constexpr bool FULL2 = (B2 * T == N1);
  static_assert(W == 8 || W == 16 || W == 32, "tile width");

  int t, c;
  __device__ __forceinline__ Col() : t((int)threadIdx.x / W), c((int)threadIdx.x % W) {}

  __device__ __forceinline__ int n2_of(int b) const { return t + T * b; }
  __device__ __forceinline__ int k1_of(int b) const { return t + T * b; }
  __device__ __forceinline__ bool ok1(int b) const { return FULL1 || (t + T * b) < N2; }
  __device__ __forceinline__ bool ok2(int b) const { return FULL2 || (t + T * b) < N1; }
  // row of the sample held in xr[b][n1] / of the frequency held in kr[b][k2]
  __device__ __forceinline__ int xrow(int b, int n1) const { return N2 * n1 + (t + T * b); }
  __device__ __forceinline__ int krow(int b, int k2) const { return (t + T * b) + N1 * k2; }

  __device__ __forceinline__ int xidx(int k1, int n2) const {
    int cc = c;
    if (W == 8) cc ^= ((k1 + n2) & 1) << 2;
    return (k1 * N2 + n2) * W + cc;
  }

  // forward (exp(-...)) transform, sample layout -> frequency layout, unnormalised.
  // tw[m] = exp(-2 pi i m / N).  One __syncthreads inside.
  __device__ __forceinline__ void fwd(float2 (&xr)[B1][N1], float2 (&kr)[B2][N2], float2* buf,
                                      const float2* tw) const {
#pragma unroll
    for (int b = 0; b < B1; ++b) {
      if (ok1(b)) {
        const int n2 = n2_of(b);
        Dft<N1, -1>::run(xr[b]);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) {
          float2 v = xr[b][k1];
          if (k1 > 0) v = cmul(v, tw[n2 * k1]);
          buf[xidx(k1, n2)] = v;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < B2; ++b) {
      if (ok2(b)) {
        const int k1 = k1_of(b);
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) kr[b][n2] = buf[xidx(k1, n2)];
        Dft<N2, -1>::run(kr[b]);
      }
    }
  }

  // inverse (exp(+...)) transform, frequency layout -> sample layout, unnormalised.
  __device__ __forceinline__ void inv(float2 (&kr)[B2][N2], float2 (&xr)[B1][N1], float2* buf,
                                      const float2* tw) const {
#pragma unroll
    for (int b = 0; b < B2; ++b) {
      if (ok2(b)) {
        const int k1 = k1_of(b);
        Dft<N2, 1>::run(kr[b]);
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) {
          float2 v = kr[b][n2];
          if (n2 > 0) v = cmulc(v, tw[n2 * k1]);
          buf[xidx(k1, n2)] = v;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < B1; ++b) {
      if (ok1(b)) {
        const int n2 = n2_of(b);
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) xr[b][k1] = buf[xidx(k1, n2)];
        Dft<N1, 1>::run(xr[b]);
      }
    }
  }
};

}  // namespace sense

// Kernel templates of the SENSE path.  Each column kernel works on one
// (column tile, frame) of an image: blockIdx.x = tile, blockIdx.y = frame.
//
//   k_fwd_col   E, first pass : S_c . x, F_y, keep sampled rows  -> tmp [F][C][L][nx]
//   k_rows      E second pass (F_x) / E^H first pass (F_x^H) on L rows per coil
//   k_adj_col   E^H second pass: zero-fill, F_y^H, conj(S_c) ., sum over c
//               (modes: plain adjoint, CG initialisation, root-sum-of-squares)
//   k_normal    E^H E column-wise: for c: S_c . p, F_y, mask, F_y^H, += conj(S_c) .
//               (CG mode: p = r + beta p prologue, Re<p,q> partials, alpha)
//   k_cg_update x += alpha p, r -= alpha q, <r,r> partials, beta / stopping test
//
// Transforms are unitary: every length-N pass scales by 1/sqrt(N).
#pragma once
#include <type_traits>

#include "common.cuh"

namespace sense {

// shared-memory bytes of the column kernels for configuration C
template <class C>
__host__ __device__ constexpr size_t col_smem_bytes_c() {
  constexpr int N = C::N;
  return sizeof(float2) * (size_t)N            // twiddles
         + 2 * sizeof(float2) * (size_t)N * C::W  // two exchange buffers
         + 32 * sizeof(double)                 // block-sum scratch
         + sizeof(short) * (size_t)N;          // line map / sampled flags
}

// Column passes (E's first pass, E^H's second pass): the length's transform
// configuration on 8-column tiles where that still fills whole warps, so a
// frame spans twice as many blocks of half the threads and several blocks
// share an SM (these passes loop over coils inside a block).
template <int N>
struct ColPass {
  using Base = typename Cfg<N>::C;
  // 384 keeps 16 columns: at 8 two 384-thread blocks would cap registers at 85
  static constexpr int W = ((Base::T * 8) % 32 == 0 && N != 384) ? 8 : Base::W;
  using C = Col<Base::T, W, typename Base::Radix>;
  static constexpr int MINB = C::THREADS <= 384 ? 2 : 1;  // resident blocks the register cap allows
};

template <int N>
__host__ __device__ constexpr size_t col_smem_bytes() {
  return col_smem_bytes_c<typename ColPass<N>::C>();
}

// Row pass (E's second pass, E^H's first): the length's transform on 8-row
// tiles where that fills whole warps (more, smaller blocks in flight for a
// pass bound by memory latency).  The staged tile has row pitch N + 1 for
// 16-row tiles and N + 2 for 8-row tiles: a half-warp then reads 16 rows (or
// 8 rows x 2 adjacent elements) on 16 distinct 8-byte bank pairs.
template <int N>
struct RowPass {
  using Base = typename Cfg<N>::C;
  static constexpr int W = (Base::T * 8) % 32 == 0 ? 8 : Base::W;
  using C = Col<Base::T, W, typename Base::Radix>;
  static constexpr int P = W == 8 ? N + 2 : N + 1;
};

template <int N>
__host__ __device__ constexpr size_t row_smem_bytes() {
  using R = RowPass<N>;
  return sizeof(float2) * (size_t)N + sizeof(float2) * (size_t)R::C::W * R::P + sizeof(float2) * (size_t)R::C::W * N +
         16;  // mbarrier of the bulk row copies
}

struct ColSmem {
  float2* tw;
  float2* buf0;
  float2* buf1;
  double* red;
  short* map;
};

// Exchange buffers for the c-th transform of a loop that runs one direction
// per iteration: with an odd number of exchanges per transform (S even) the
// pair is swapped every iteration, so no buffer is written while another
// thread may still read it.
template <class C>
struct BufPair {
  float2* b[2];
  __device__ __forceinline__ BufPair(float2* b0, float2* b1, int iter) {
    const bool swap = ((C::S % 2) == 0) && (iter & 1);
    b[0] = swap ? b1 : b0;
    b[1] = swap ? b0 : b1;
  }
};

template <class C>
__device__ __forceinline__ ColSmem col_smem_c(unsigned char* base) {
  constexpr int N = C::N;
  ColSmem s;
  s.tw = reinterpret_cast<float2*>(base);
  s.buf0 = s.tw + N;
  s.buf1 = s.buf0 + N * C::W;
  s.red = reinterpret_cast<double*>(s.buf1 + N * C::W);
  s.map = reinterpret_cast<short*>(s.red + 32);
  return s;
}

template <int N>
__device__ __forceinline__ ColSmem col_smem(unsigned char* base) {
  return col_smem_c<typename ColPass<N>::C>(base);
}

// Centred k-space (DC at n/2): F_c = (-1)^(n/2) D F D with D = diag((-1)^i),
// so the kernels keep the uncentred transforms and flip signs at their loads
// and stores: image pixels by (-1)^(y+x), k-space rows by (-1)^ky, row
// elements by (-1)^kx times the constant (-1)^(ny/2 + nx/2).
__device__ __forceinline__ float2 negate_if(float2 v, bool neg) {
  return neg ? make_float2(-v.x, -v.y) : v;
}

// Copy the twiddles and build map[row] = index of `row` in this frame's line
// list, or -1 if the row is not sampled.  Out-of-range or unordered lines are
// skipped and flagged.
template <int N, int THREADS>
__device__ __forceinline__ void load_tw_and_linemap(const ColSmem& s, const float2* tw, const int* ln, int L,
                                                   int* err) {
  for (int i = threadIdx.x; i < N; i += THREADS) {
    s.tw[i] = tw[i];
    s.map[i] = -1;
  }
  __syncthreads();
  for (int l = threadIdx.x; l < L; l += THREADS) {
    const int v = __ldg(ln + l);
    const bool good = v >= 0 && v < N && (l == 0 || __ldg(ln + l - 1) < v);
    if (good)
      s.map[v] = (short)l;
    else
      atomicOr(err, ERR_LINES);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// E, column pass
// ---------------------------------------------------------------------------
template <class St>
struct FwdColArgs {
  const float2* x;              // [F][N][nx]
  const typename St::T* S;      // [C][N][nx]
  const int* lines;             // [F][L]
  float2* tmp;                  // [F][C][L][nx]
  const float2* tw;
  int nx, coils, L;
  int centred;                  // 1: centred k-space (image and k-space row signs)
  int* err;
};

template <int N, class St, int TH = ColPass<N>::C::THREADS>
__global__ void __launch_bounds__(TH, ColPass<N>::MINB) k_fwd_col(FwdColArgs<St> a) {
  using C = typename ColPass<N>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ColSmem s = col_smem<N>(smem_raw);
  const int f = blockIdx.y;
  const C col;
  const int x = blockIdx.x * C::W + col.c;
  const bool xin = x < a.nx;
  load_tw_and_linemap<N, C::THREADS>(s, a.tw, a.lines + (size_t)f * a.L, a.L, a.err);
  const size_t img = (size_t)N * a.nx;
  const float scale = rsqrtf((float)N);

  float2 xv[C::J0][C::R0];
#pragma unroll
  for (int j = 0; j < C::J0; ++j)
#pragma unroll
    for (int n = 0; n < C::R0; ++n)
      xv[j][n] = (col.ok0(j) && xin) ? negate_if(__ldg(a.x + f * img + (size_t)col.xrow(j, n) * a.nx + x),
                                                 a.centred && ((col.xrow(j, n) + x) & 1))
                                      : make_float2(0.f, 0.f);

#pragma unroll 1
  for (int c = 0; c < a.coils; ++c) {
    float2 xr[C::J0][C::R0];
    float2 kr[C::JL][C::RL];
#pragma unroll
    for (int j = 0; j < C::J0; ++j)
#pragma unroll
      for (int n = 0; n < C::R0; ++n) {
        float2 sv = make_float2(0.f, 0.f);
        if (col.ok0(j) && xin) sv = St::ld(a.S, c * img + (size_t)col.xrow(j, n) * a.nx + x);
        xr[j][n] = cmul(sv, xv[j][n]);
      }
    const BufPair<C> bp(s.buf0, s.buf1, c);
    col.fwd(xr, kr, bp.b, s.tw);
    float2* dst = a.tmp + ((size_t)f * a.coils + c) * a.L * a.nx;
#pragma unroll
    for (int j = 0; j < C::JL; ++j)
#pragma unroll
      for (int m = 0; m < C::RL; ++m) {
        if (col.okL(j) && xin) {
          const int l = s.map[col.krow(j, m)];
          if (l >= 0)
            dst[(size_t)l * a.nx + x] = negate_if(cscale(kr[j][m], scale), a.centred && (col.krow(j, m) & 1));
        }
      }
  }
}

// ---------------------------------------------------------------------------
// Row pass: W rows of length N per block, transformed along the row.
// DIR = -1: forward (E second pass), FP32 in, storage out.
// DIR = +1: inverse (E^H first pass), storage in, FP32 out.
// ---------------------------------------------------------------------------
template <class InT, class OutT>
struct RowArgs {
  const InT* in;
  OutT* out;
  const float2* tw;
  long rows;
  int centred;  // 1: k-space elements times cs (-1)^kx (inverse: on input; forward: on output)
  float cs;     // (-1)^(ny/2 + nx/2)
  int* err;     // error word (ERR_TIMEOUT from a bulk copy that never landed); may be NULL
};

template <int N, int DIR, class InSt, class OutSt, int TH = RowPass<N>::C::THREADS>
__global__ void __launch_bounds__(TH)
    k_rows(RowArgs<typename InSt::T, typename OutSt::T> a) {
  using C = typename RowPass<N>::C;
  constexpr int P = RowPass<N>::P;  // padded row pitch (conflict-free column access)
  // Complex64 rows move between global and shared memory as 1D bulk copies,
  // one per row, instead of through registers: with N even and the pitch
  // N + 2, every global row and every shared row starts 16-byte aligned
  // when the base pointer is (checked at run time; otherwise the threads copy).
  constexpr bool kBulkIn = std::is_same<typename InSt::T, float2>::value && P == N + 2;
  constexpr bool kBulkOut = std::is_same<typename OutSt::T, float2>::value && P == N + 2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* tile = tw + N;
  float2* bufs[2] = {tile, tile + C::W * P};  // the tile doubles as the first exchange buffer
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + row_smem_bytes<N>() - 16);
  const C col;
  const long r0 = (long)blockIdx.x * C::W;
  const int nrows = (int)((a.rows - r0) < (long)C::W ? (a.rows - r0) : (long)C::W);
  const bool bulk_in = kBulkIn && (reinterpret_cast<uintptr_t>(a.in) & 15u) == 0;
  const bool bulk_out = kBulkOut && (reinterpret_cast<uintptr_t>(a.out) & 15u) == 0;
  constexpr unsigned kRowBytes = (unsigned)(sizeof(float2) * N);
  bool landed = true;  // false if the bulk row copies never completed: the block then stores nothing
  if (bulk_in) {
    if (threadIdx.x == 0) {
      mbar_init(bar, 1);
      mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      mbar_arrive_expect_tx(bar, kRowBytes * (unsigned)nrows);
      for (int rr = 0; rr < nrows; ++rr)
        bulk_load(tile + rr * P, reinterpret_cast<const float2*>(a.in) + (size_t)(r0 + rr) * N, kRowBytes, bar);
    }
    for (int i = threadIdx.x; i < N; i += C::THREADS) tw[i] = a.tw[i];
    if (!mbar_wait(bar, 0)) {  // never expected; flag it and let the copies land before going on
      if (threadIdx.x == 0 && a.err) atomicOr(a.err, ERR_TIMEOUT);
      landed = mbar_wait(bar, 0);
    }
  } else {
    // every load of the tile is issued before the first shared store
    constexpr int PER = (C::W * N + C::THREADS - 1) / C::THREADS;
    float2 v[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int i = (int)threadIdx.x + k * C::THREADS;
      const int rr = i / N, e = i - rr * N;
      v[k] = (i < C::W * N && r0 + rr < a.rows) ? InSt::ld(a.in, (size_t)(r0 + rr) * N + e) : make_float2(0.f, 0.f);
      if (DIR > 0 && a.centred) v[k] = cscale(v[k], (e & 1) ? -a.cs : a.cs);
    }
    for (int i = threadIdx.x; i < N; i += C::THREADS) tw[i] = a.tw[i];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int i = (int)threadIdx.x + k * C::THREADS;
      const int rr = i / N, e = i - rr * N;
      if (i < C::W * N) tile[rr * P + e] = v[k];
    }
  }
  if (!__syncthreads_and(landed)) return;  // uniform: the tile never arrived (ERR_TIMEOUT raised)
  const float scale = rsqrtf((float)N);
  float2 xr[C::J0][C::R0];
  float2 kr[C::JL][C::RL];
  float2* row = tile + col.c * P;
  if (DIR < 0) {
#pragma unroll
    for (int j = 0; j < C::J0; ++j)
#pragma unroll
      for (int n = 0; n < C::R0; ++n) xr[j][n] = col.ok0(j) ? row[col.xrow(j, n)] : make_float2(0.f, 0.f);
    __syncthreads();  // the tile becomes the exchange buffer
    col.fwd(xr, kr, bufs, tw);
    __syncthreads();
    // centred k-space: with the bulk store the signs go on here, not at the global store
    const bool sign_here = bulk_out && a.centred;
#pragma unroll
    for (int j = 0; j < C::JL; ++j)
#pragma unroll
      for (int m = 0; m < C::RL; ++m)
        if (col.okL(j)) {
          const int e = col.krow(j, m);
          row[e] = cscale(kr[j][m], sign_here ? ((e & 1) ? -scale * a.cs : scale * a.cs) : scale);
        }
  } else {
    const bool sign_here = bulk_in && a.centred;  // the bulk load did not apply the k-space signs
#pragma unroll
    for (int j = 0; j < C::JL; ++j)
#pragma unroll
      for (int m = 0; m < C::RL; ++m) {
        const int e = col.krow(j, m);
        kr[j][m] = col.okL(j) ? row[e] : make_float2(0.f, 0.f);
        if (sign_here) kr[j][m] = cscale(kr[j][m], (e & 1) ? -a.cs : a.cs);
      }
    __syncthreads();
    col.inv(kr, xr, bufs, tw);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < C::J0; ++j)
#pragma unroll
      for (int n = 0; n < C::R0; ++n)
        if (col.ok0(j)) row[col.xrow(j, n)] = cscale(xr[j][n], scale);
  }
  if (bulk_out) {
    fence_proxy_async_smem();  // this thread's shared writes, before the bulk engine reads them
    __syncthreads();
    if ((int)threadIdx.x < nrows) {
      bulk_store(reinterpret_cast<float2*>(a.out) + (size_t)(r0 + threadIdx.x) * N, tile + threadIdx.x * P,
                 kRowBytes);
      bulk_commit_wait_read();
    }
    return;
  }
  __syncthreads();
  {
    constexpr int PER = (C::W * N + C::THREADS - 1) / C::THREADS;
    float2 v[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int i = (int)threadIdx.x + k * C::THREADS;
      const int rr = i / N, e = i - rr * N;
      v[k] = i < C::W * N ? tile[rr * P + e] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int i = (int)threadIdx.x + k * C::THREADS;
      const int rr = i / N, e = i - rr * N;
      if (DIR < 0 && a.centred) v[k] = cscale(v[k], (e & 1) ? -a.cs : a.cs);
      if (i < C::W * N && r0 + rr < a.rows) OutSt::st(a.out, (size_t)(r0 + rr) * N + e, v[k]);
    }
  }
}

// Row pass over complex64 rows in and out, persistent: each block loops over
// row tiles (blockIdx.x, + gridDim.x, ...).  While it transforms one tile,
// the bulk-copy engine brings the next tile's rows into the other of two
// tile buffers, so the HBM latency of a block's loads hides behind its own
// arithmetic.  Results go back by per-row bulk stores from the tile.  The
// launcher uses it when both pointers are 16-byte aligned (rows then start
// 16-byte aligned, N being even) and the pitch is N + 2.
template <int N>
__host__ __device__ constexpr size_t row_bulk_smem_bytes() {
  using R = RowPass<N>;
  return sizeof(float2) * ((size_t)N + 2 * (size_t)R::C::W * R::P + (size_t)R::C::W * N) + 16;
}

template <int N, int DIR, int TH = RowPass<N>::C::THREADS>
__global__ void __launch_bounds__(TH) k_rows_bulk(RowArgs<float2, float2> a) {
  using C = typename RowPass<N>::C;
  constexpr int P = RowPass<N>::P;
  static_assert(P == N + 2, "bulk row copies need the 16-byte row pitch N + 2");
  constexpr unsigned kRowBytes = (unsigned)(sizeof(float2) * N);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* const tile0 = tw + N;  // picked with selects: a run-time index would put a pointer array in local memory
  float2* const tile1 = tw + N + C::W * P;
  float2* buf1 = tw + N + 2 * C::W * P;
  uint64_t* bar = reinterpret_cast<uint64_t*>(buf1 + C::W * N);  // one per tile buffer
  const long ntiles = (a.rows + C::W - 1) / C::W;
  const C col;
  // thread 0: arm bar[b] and copy the rows of tile t into buffer b
  auto fetch = [&](long t, int b) {
    const long r0 = t * C::W;
    const int nrows = (int)((a.rows - r0) < (long)C::W ? (a.rows - r0) : (long)C::W);
    mbar_arrive_expect_tx(bar + b, kRowBytes * (unsigned)nrows);
    float2* dst = b ? tile1 : tile0;
    for (int rr = 0; rr < nrows; ++rr) bulk_load(dst + rr * P, a.in + (size_t)(r0 + rr) * N, kRowBytes, bar + b);
  };
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    mbar_init(bar + 1, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && (long)blockIdx.x < ntiles) fetch(blockIdx.x, 0);
  for (int i = threadIdx.x; i < N; i += C::THREADS) tw[i] = a.tw[i];
  __syncthreads();
  const float scale = rsqrtf((float)N);
  int it = 0;
  for (long t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
    const int cur = it & 1;
    const long r0 = t * C::W;
    const int nrows = (int)((a.rows - r0) < (long)C::W ? (a.rows - r0) : (long)C::W);
    // the other buffer's last stores have read it (waited below, then a barrier)
    if (threadIdx.x == 0 && t + gridDim.x < ntiles) fetch(t + gridDim.x, cur ^ 1);
    const unsigned parity = (unsigned)(it >> 1) & 1u;
    bool landed = true;
    if (!mbar_wait(bar + cur, parity)) {  // never expected; flag it and let the copies land
      if (threadIdx.x == 0 && a.err) atomicOr(a.err, ERR_TIMEOUT);
      landed = mbar_wait(bar + cur, parity);
    }
    // a tile that never arrived is skipped by the whole block (its rows keep their contents)
    const bool skip = !__syncthreads_and(landed);
    float2* tile = cur ? tile1 : tile0;
    float2* bufs[2] = {tile, buf1};  // the tile doubles as the first exchange buffer
    float2* row = tile + col.c * P;
    float2 xr[C::J0][C::R0];
    float2 kr[C::JL][C::RL];
    if (DIR < 0) {
#pragma unroll
      for (int j = 0; j < C::J0; ++j)
#pragma unroll
        for (int n = 0; n < C::R0; ++n) xr[j][n] = col.ok0(j) ? row[col.xrow(j, n)] : make_float2(0.f, 0.f);
      __syncthreads();
      col.fwd(xr, kr, bufs, tw);
      __syncthreads();
#pragma unroll
      for (int j = 0; j < C::JL; ++j)
#pragma unroll
        for (int m = 0; m < C::RL; ++m)
          if (col.okL(j)) {
            const int e = col.krow(j, m);  // centred k-space: sign (-1)^kx on the output
            row[e] = cscale(kr[j][m], a.centred ? ((e & 1) ? -scale * a.cs : scale * a.cs) : scale);
          }
    } else {
#pragma unroll
      for (int j = 0; j < C::JL; ++j)
#pragma unroll
        for (int m = 0; m < C::RL; ++m) {
          const int e = col.krow(j, m);  // centred k-space: sign (-1)^kx on the input
          kr[j][m] = col.okL(j) ? row[e] : make_float2(0.f, 0.f);
          if (a.centred) kr[j][m] = cscale(kr[j][m], (e & 1) ? -a.cs : a.cs);
        }
      __syncthreads();
      col.inv(kr, xr, bufs, tw);
      __syncthreads();
#pragma unroll
      for (int j = 0; j < C::J0; ++j)
#pragma unroll
        for (int n = 0; n < C::R0; ++n)
          if (col.ok0(j)) row[col.xrow(j, n)] = cscale(xr[j][n], scale);
    }
    fence_proxy_async_smem();  // this thread's shared writes, before the bulk engine reads them
    __syncthreads();
    if (!skip && (int)threadIdx.x < nrows) {
      bulk_store(a.out + (size_t)(r0 + threadIdx.x) * N, tile + threadIdx.x * P, kRowBytes);
      bulk_commit_wait_read();
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// E^H, column pass.  MODE 0: x = sum_c conj(S_c) F_y^H(...)
//                    MODE 1: same, written as CG start r = p = b, x = 0, rho0
//                    MODE 2: root sum of squares over coils (S unused)
// ---------------------------------------------------------------------------
template <class St>
struct AdjColArgs {
  const float2* tmp;          // [F][C][L][nx], rows already inverse-transformed
  const typename St::T* S;    // [C][N][nx]
  const int* lines;
  const float2* tw;
  float2* x;                  // MODE 0: output; MODE 1: zeroed
  float2* r;                  // MODE 1
  float2* p;                  // MODE 1
  float* rss;                 // MODE 2
  int nx, coils, L, tiles;
  int centred;                // 1: k-space rows by (-1)^ky; MODE 0 output by (-1)^(y+x)
  int* err;
  CgState cg;
};

template <int N, class St, int MODE, int TH = ColPass<N>::C::THREADS>
__global__ void __launch_bounds__(TH, ColPass<N>::MINB) k_adj_col(AdjColArgs<St> a) {
  using C = typename ColPass<N>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ColSmem s = col_smem<N>(smem_raw);
  const int f = blockIdx.y;
  const C col;
  const int x = blockIdx.x * C::W + col.c;
  const bool xin = x < a.nx;
  load_tw_and_linemap<N, C::THREADS>(s, a.tw, a.lines + (size_t)f * a.L, a.L, a.err);
  const size_t img = (size_t)N * a.nx;

  float2 acc[C::J0][C::R0], accl[C::J0][C::R0];  // compensated coil sum (MODE 0, 1)
  float accr[C::J0][C::R0];
#pragma unroll
  for (int j = 0; j < C::J0; ++j)
#pragma unroll
    for (int n = 0; n < C::R0; ++n) {
      acc[j][n] = make_float2(0.f, 0.f);
      accl[j][n] = make_float2(0.f, 0.f);
      accr[j][n] = 0.f;
    }

  // With blocks of up to 256 threads and at most 24 values per thread per
  // side (registers to spare at two blocks per SM), coil c + 1's k-space
  // values and maps are loaded into registers before coil c is transformed,
  // so their latency overlaps the transform.
  constexpr bool PREFETCH = C::THREADS <= 256 && C::J0 * C::R0 + C::JL * C::RL <= 24;
  auto load_k = [&](int c, float2 (&kv)[C::JL][C::RL]) {
    const float2* src = a.tmp + ((size_t)f * a.coils + c) * a.L * a.nx;
#pragma unroll
    for (int j = 0; j < C::JL; ++j)
#pragma unroll
      for (int m = 0; m < C::RL; ++m) {
        const int l = (col.okL(j) && xin) ? (int)s.map[col.krow(j, m)] : -1;
        kv[j][m] = l >= 0 ? __ldg(src + (size_t)l * a.nx + x) : make_float2(0.f, 0.f);
      }
  };
  auto load_s = [&](int c, float2 (&sv)[C::J0][C::R0]) {
#pragma unroll
    for (int j = 0; j < C::J0; ++j)
#pragma unroll
      for (int n = 0; n < C::R0; ++n)
        sv[j][n] = (MODE != 2 && col.ok0(j) && xin) ? St::ld(a.S, c * img + (size_t)col.xrow(j, n) * a.nx + x)
                                                    : make_float2(0.f, 0.f);
  };
  // Register twiddles (loaded once, reused by every coil) where the register
  // budget has room: RSS mode, or a cap of at least 160 registers per thread.
  constexpr bool REG_TW = MODE == 2 || 65536 / (C::THREADS * ColPass<N>::MINB) >= 160;
  typename C::Tw0 w0;
  if constexpr (REG_TW) w0 = col.load_tw0(s.tw);
  float2 knext[C::JL][C::RL];
  float2 snext[C::J0][C::R0];
  if (PREFETCH && a.coils > 0) {
    load_k(0, knext);
    load_s(0, snext);
  }
#pragma unroll 1
  for (int c = 0; c < a.coils; ++c) {
    float2 xr[C::J0][C::R0];
    float2 kr[C::JL][C::RL];
    float2 sv[C::J0][C::R0];
    if constexpr (PREFETCH) {
#pragma unroll
      for (int j = 0; j < C::JL; ++j)
#pragma unroll
        for (int m = 0; m < C::RL; ++m) kr[j][m] = knext[j][m];
#pragma unroll
      for (int j = 0; j < C::J0; ++j)
#pragma unroll
        for (int n = 0; n < C::R0; ++n) sv[j][n] = snext[j][n];
      if (c + 1 < a.coils) {
        load_k(c + 1, knext);
        load_s(c + 1, snext);
      }
    } else {
      load_k(c, kr);
      load_s(c, sv);
    }
    if (a.centred) {  // k-space rows by (-1)^ky, once the values are in registers
#pragma unroll
      for (int j = 0; j < C::JL; ++j)
#pragma unroll
        for (int m = 0; m < C::RL; ++m) kr[j][m] = negate_if(kr[j][m], col.krow(j, m) & 1);
    }
    const BufPair<C> bp(s.buf0, s.buf1, c);
    if constexpr (REG_TW)
      col.inv(kr, xr, bp.b, s.tw, w0);
    else
      col.inv(kr, xr, bp.b, s.tw);
#pragma unroll
    for (int j = 0; j < C::J0; ++j)
#pragma unroll
      for (int n = 0; n < C::R0; ++n) {
        if (MODE == 2)
          accr[j][n] = fmaf(xr[j][n].x, xr[j][n].x, fmaf(xr[j][n].y, xr[j][n].y, accr[j][n]));
        else
          csum_fma_conj(acc[j][n], accl[j][n], sv[j][n], xr[j][n]);
      }
  }

  const float scale = rsqrtf((float)N);
  float part = 0.f;
#pragma unroll
  for (int j = 0; j < C::J0; ++j)
#pragma unroll
    for (int n = 0; n < C::R0; ++n) {
      if (!(col.ok0(j) && xin)) continue;
      const size_t idx = f * img + (size_t)col.xrow(j, n) * a.nx + x;
      if (MODE == 2) {
        a.rss[idx] = sqrtf(accr[j][n] * (1.0f / (float)N));
      } else {
        const float2 v = cscale(csum_value(acc[j][n], accl[j][n]), scale);
        if (MODE == 0) {
          a.x[idx] = negate_if(v, a.centred && ((col.xrow(j, n) + x) & 1));
        } else {
          a.r[idx] = v;
          a.p[idx] = v;
          a.x[idx] = make_float2(0.f, 0.f);
          part = fmaf(v.x, v.x, fmaf(v.y, v.y, part));
        }
      }
    }

  if (MODE == 1) {
    const double tot = block_sum<C::THREADS>((double)part, s.red);
    const CgState& g = a.cg;
    double* slot = g.part + (size_t)f * g.part_stride + blockIdx.x;
    if (publish_and_arrive(tot, slot, g.counter + f, (unsigned)a.tiles)) {
      const double rho = ordered_sum(g.part + (size_t)f * g.part_stride, a.tiles);
      g.counter[f] = 0u;
      g.rho[f] = rho;
      g.rho0[f] = rho;
      g.iters[f] = 0;
      g.beta[f] = 0.0;
      g.alpha[f] = 0.0;
      if (rho > 0.0 && isfinite(rho)) {
        g.active[f] = 1;
        g.outcome[f] = CG_RUNNING;
        g.resid[f] = 1.0;
        atomicAdd(g.live, 1);
      } else {  // b = 0 (converged at once) or not finite (NaN/Inf input: breakdown, residual NaN)
        g.active[f] = 0;
        g.outcome[f] = (rho == 0.0) ? CG_CONVERGED : CG_BREAKDOWN;
        g.resid[f] = (rho == 0.0) ? 0.0 : rho - rho;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// E^H E, column-wise, for one (frame, column tile).  Used by k_normal (one
// launch per operator application) and by the persistent CG kernel.
//   CG=false: out = E^H E x.
//   CG=true : p_k = r + beta p_{k-1} formed on the fly when p_update (read
//             from p_src, written to p_dst), q = E^H E p_k; returns this
//             thread's share of Re<p_k, q> (FP32 over its own elements).
// Inputs that other blocks of the same launch may have written are read
// through L2 (ld.global.cg), and outputs are written the same way.
// ---------------------------------------------------------------------------
struct NormalTile {
  const float2* x;      // CG=false input, frame base
  float2* out;          // CG=false output, frame base
  const float2* p_src;  // CG=true, frame base
  float2* p_dst;        // CG=true, frame base
  const float2* r;      // CG=true, frame base
  float2* q;            // CG=true, frame base
  const void* S;        // maps [C][N][nx], storage type
  int nx, coils, tile, p_update;
  int centred;          // CG=false: x and out signed by (-1)^(y+x)
  float beta;
  float lambda;         // CG=true: Tikhonov weight, q = E^H E p + lambda p
  // CG=true, frames coupled in time (lambda_t > 0): q += lambda_t (2 p - p_prev - p_next)
  // with the neighbouring frames' current directions formed on the fly,
  // p_nb = r_nb + beta ps_nb (or ps_nb itself when !p_update)
  float lambda_t;
  const float2 *r_prev, *r_next, *ps_prev, *ps_next;
};

// The temporal term lambda_t (2 p - p_prev - p_next) at image index idx.
__device__ __forceinline__ float2 neighbour_direction(const NormalTile& a, const float2* ps, const float2* r,
                                                      size_t idx) {
  float2 v = __ldcg(ps + idx);
  if (a.p_update) {
    const float2 rv = __ldcg(r + idx);
    v = make_float2(fmaf(a.beta, v.x, rv.x), fmaf(a.beta, v.y, rv.y));
  }
  return v;
}
__device__ __forceinline__ float2 temporal_term(const NormalTile& a, size_t idx, float2 p) {
  const float2 pp = neighbour_direction(a, a.ps_prev, a.r_prev, idx);
  const float2 pn = neighbour_direction(a, a.ps_next, a.r_next, idx);
  return make_float2(a.lambda_t * (2.f * p.x - pp.x - pn.x), a.lambda_t * (2.f * p.y - pp.y - pn.y));
}

template <class C, class St, bool CG>
__device__ __forceinline__ float normal_tile(const NormalTile& a, const ColSmem& s, unsigned keep) {
  constexpr int N = C::N;
  const C col;
  const int x = a.tile * C::W + col.c;
  const bool xin = x < a.nx;
  const size_t img = (size_t)N * a.nx;
  float2 p[C::J0][C::R0], q[C::J0][C::R0], ql[C::J0][C::R0];  // q: compensated coil sum
#pragma unroll
  for (int j = 0; j < C::J0; ++j)
#pragma unroll
    for (int n = 0; n < C::R0; ++n) {
      float2 v = make_float2(0.f, 0.f);
      if (col.ok0(j) && xin) {
        const size_t idx = (size_t)col.xrow(j, n) * a.nx + x;
        if (CG) {
          v = __ldcg(a.p_src + idx);
          if (a.p_update) {
            const float2 rv = __ldcg(a.r + idx);
            v = make_float2(fmaf(a.beta, v.x, rv.x), fmaf(a.beta, v.y, rv.y));
            __stcg(a.p_dst + idx, v);
          }
        } else {
          v = negate_if(__ldg(a.x + idx), a.centred && ((col.xrow(j, n) + x) & 1));
        }
      }
      p[j][n] = v;
      q[j][n] = make_float2(0.f, 0.f);
      ql[j][n] = make_float2(0.f, 0.f);
    }

  float2* bufs[2] = {s.buf0, s.buf1};
  const typename St::T* Sc = static_cast<const typename St::T*>(a.S) + x;
#pragma unroll 1
  for (int c = 0; c < a.coils; ++c, Sc += img) {
    float2 xr[C::J0][C::R0];
    float2 kr[C::JL][C::RL];
#pragma unroll
    for (int j = 0; j < C::J0; ++j)
#pragma unroll
      for (int n = 0; n < C::R0; ++n) {
        float2 sv = make_float2(0.f, 0.f);
        if (col.ok0(j) && xin) sv = St::ld(Sc, (size_t)col.xrow(j, n) * a.nx);
        xr[j][n] = cmul(sv, p[j][n]);
      }
    col.fwd(xr, kr, bufs, s.tw);
#pragma unroll
    for (int j = 0; j < C::JL; ++j)
#pragma unroll
      for (int m = 0; m < C::RL; ++m)
        if (!((keep >> (j * C::RL + m)) & 1u)) kr[j][m] = make_float2(0.f, 0.f);
    col.inv(kr, xr, bufs, s.tw);
#pragma unroll
    for (int j = 0; j < C::J0; ++j)
#pragma unroll
      for (int n = 0; n < C::R0; ++n) {
        float2 sv = make_float2(0.f, 0.f);
        if (col.ok0(j) && xin) sv = St::ld(Sc, (size_t)col.xrow(j, n) * a.nx);
        csum_fma_conj(q[j][n], ql[j][n], sv, xr[j][n]);
      }
  }

  const float invN = 1.0f / (float)N;  // the two unitary transforms' 1/sqrt(N) each
  float part = 0.f;
#pragma unroll
  for (int j = 0; j < C::J0; ++j)
#pragma unroll
    for (int n = 0; n < C::R0; ++n) {
      if (!(col.ok0(j) && xin)) continue;
      const size_t idx = (size_t)col.xrow(j, n) * a.nx + x;
      float2 qv = cscale(csum_value(q[j][n], ql[j][n]), invN);
      if (CG) {
        qv = make_float2(fmaf(a.lambda, p[j][n].x, qv.x), fmaf(a.lambda, p[j][n].y, qv.y));
        if (a.lambda_t != 0.f) qv = cadd(qv, temporal_term(a, idx, p[j][n]));
        __stcg(a.q + idx, qv);
        part = fmaf(p[j][n].x, qv.x, fmaf(p[j][n].y, qv.y, part));
      } else {
        a.out[idx] = negate_if(qv, a.centred && ((col.xrow(j, n) + x) & 1));
      }
    }
  return part;
}

// One bit per frequency row this thread holds: set if the row is sampled.
template <class C>
__device__ __forceinline__ unsigned sampled_bits(const short* map) {
  static_assert(C::JL * C::RL <= 32, "mask bits");
  const C col;
  unsigned keep = 0u;
#pragma unroll
  for (int j = 0; j < C::JL; ++j)
#pragma unroll
    for (int m = 0; m < C::RL; ++m)
      if (col.okL(j) && map[col.krow(j, m)] >= 0) keep |= 1u << (j * C::RL + m);
  return keep;
}

// line map of a frame: map[row] = index in the frame's line list, or -1
// (The first round of line loads is issued before the map is cleared, so
// its latency overlaps the clearing and the barrier.)
template <int N, int THREADS>
__device__ __forceinline__ void build_linemap(short* map, const int* ln, int L, int* err) {
  const int l0 = (int)threadIdx.x;
  int v0 = 0, u0 = -1;
  if (l0 < L) {
    v0 = __ldg(ln + l0);
    if (l0 > 0) u0 = __ldg(ln + l0 - 1);
  }
  for (int i = threadIdx.x; i < N; i += THREADS) map[i] = -1;
  __syncthreads();
  for (int l = l0; l < L; l += THREADS) {
    const int v = l == l0 ? v0 : __ldg(ln + l);
    const int u = l == l0 ? u0 : __ldg(ln + l - 1);  // l > 0 unless l == l0 == 0
    const bool good = v >= 0 && v < N && (l == 0 || u < v);
    if (good)
      map[v] = (short)l;
    else
      atomicOr(err, ERR_LINES);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// TMA-staged variant of normal_tile (CG mode): the maps of each coil arrive
// as one [N][W] tile in shared memory by a 2D bulk tensor copy, double
// buffered.  Fill i of the block goes to buffer i & 1 and completes phase
// (i >> 1) & 1 of that buffer's mbarrier.  The caller has issued the fill of
// this tile's first coil (fill index nfill); the fill of coil c + 1 is issued
// after coil c's forward transform, whose barriers guarantee that every
// thread has finished reading that buffer two coils back.
// ---------------------------------------------------------------------------
template <class C, class St>
struct SStage {
  typename St::T* buf[2];
  uint64_t* bar;  // [2]
  const void* tmap;
  static constexpr unsigned BYTES = (unsigned)(C::N * C::W * sizeof(typename St::T));
  // thread 0: copy the [N][W] map tile of coil c, columns tile*W.., into fill slot i
  __device__ __forceinline__ void issue(unsigned i, int tile, int c) const {
    typename St::T* dst = (i & 1) ? buf[1] : buf[0];  // constant indices keep the struct in registers
    uint64_t* b = bar + (i & 1);
    tmap_acquire(tmap);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(b, BYTES);
    if constexpr (C::N <= 256) {
      tma_load_2d(dst, tmap, tile * C::W, c * C::N, b);
    } else {
      tma_load_2d(dst, tmap, tile * C::W, c * C::N, b);
      tma_load_2d(dst + (C::N / 2) * C::W, tmap, tile * C::W, c * C::N + C::N / 2, b);
    }
  }
};

template <class C, class St>
__device__ __forceinline__ float normal_tile_tma(const NormalTile& a, const ColSmem& s, unsigned keep,
                                                 const SStage<C, St>& sg, unsigned nfill, int* err,
                                                 const int* lines = nullptr, int L = 0) {
  constexpr int N = C::N;
  const C col;
  const int x = a.tile * C::W + col.c;
  const bool xin = x < a.nx;
  float2 p[C::J0][C::R0], q[C::J0][C::R0], ql[C::J0][C::R0];  // q: compensated coil sum
  {
    // every load first, so their latencies overlap (and, given `lines`, the
    // frame's line map is built while they are in flight)
    float2 rv[C::J0][C::R0];
#pragma unroll
    for (int j = 0; j < C::J0; ++j)
#pragma unroll
      for (int n = 0; n < C::R0; ++n) {
        p[j][n] = make_float2(0.f, 0.f);
        rv[j][n] = make_float2(0.f, 0.f);
        if (col.ok0(j) && xin) {
          const size_t idx = (size_t)col.xrow(j, n) * a.nx + x;
          p[j][n] = __ldcg(a.p_src + idx);
          if (a.p_update) rv[j][n] = __ldcg(a.r + idx);
        }
      }
    if (lines) {
      build_linemap<N, C::THREADS>(s.map, lines, L, err);
      keep = sampled_bits<C>(s.map);
    }
#pragma unroll
    for (int j = 0; j < C::J0; ++j)
#pragma unroll
      for (int n = 0; n < C::R0; ++n) {
        if (col.ok0(j) && xin && a.p_update) {
          p[j][n] = make_float2(fmaf(a.beta, p[j][n].x, rv[j][n].x), fmaf(a.beta, p[j][n].y, rv[j][n].y));
          __stcg(a.p_dst + (size_t)col.xrow(j, n) * a.nx + x, p[j][n]);
        }
        q[j][n] = make_float2(0.f, 0.f);
        ql[j][n] = make_float2(0.f, 0.f);
      }
  }

  float2* bufs[2] = {s.buf0, s.buf1};
#pragma unroll 1
  for (int c = 0; c < a.coils; ++c) {
    const unsigned i = nfill + (unsigned)c;
    if (!mbar_wait(sg.bar + (i & 1), (i >> 1) & 1u)) atomicOr(err, ERR_TIMEOUT);
    const typename St::T* sb = (i & 1) ? sg.buf[1] : sg.buf[0];
    float2 xr[C::J0][C::R0];
    float2 kr[C::JL][C::RL];
#pragma unroll
    for (int j = 0; j < C::J0; ++j)
#pragma unroll
      for (int n = 0; n < C::R0; ++n) {
        const float2 sv = col.ok0(j) ? St::lds(sb, col.xrow(j, n) * C::W + col.c) : make_float2(0.f, 0.f);
        xr[j][n] = cmul(sv, p[j][n]);
      }
    col.fwd(xr, kr, bufs, s.tw);
    if (threadIdx.x == 0 && c + 1 < a.coils) sg.issue(i + 1, a.tile, c + 1);
#pragma unroll
    for (int j = 0; j < C::JL; ++j)
#pragma unroll
      for (int m = 0; m < C::RL; ++m)
        if (!((keep >> (j * C::RL + m)) & 1u)) kr[j][m] = make_float2(0.f, 0.f);
    col.inv(kr, xr, bufs, s.tw);
#pragma unroll
    for (int j = 0; j < C::J0; ++j)
#pragma unroll
      for (int n = 0; n < C::R0; ++n) {
        const float2 sv = col.ok0(j) ? St::lds(sb, col.xrow(j, n) * C::W + col.c) : make_float2(0.f, 0.f);
        csum_fma_conj(q[j][n], ql[j][n], sv, xr[j][n]);
      }
  }

  const float invN = 1.0f / (float)N;
  float part = 0.f;
#pragma unroll
  for (int j = 0; j < C::J0; ++j)
#pragma unroll
    for (int n = 0; n < C::R0; ++n) {
      if (!(col.ok0(j) && xin)) continue;
      const size_t idx = (size_t)col.xrow(j, n) * a.nx + x;
      float2 qv = cscale(csum_value(q[j][n], ql[j][n]), invN);
      qv = make_float2(fmaf(a.lambda, p[j][n].x, qv.x), fmaf(a.lambda, p[j][n].y, qv.y));
      if (a.lambda_t != 0.f) qv = cadd(qv, temporal_term(a, idx, p[j][n]));
      __stcg(a.q + idx, qv);
      part = fmaf(p[j][n].x, qv.x, fmaf(p[j][n].y, qv.y, part));
    }
  return part;
}

// ---------------------------------------------------------------------------
// Lane-major tiles (WCol configurations): each column is transformed by the
// lanes of one warp, so the coil loop has no block-wide barrier.
//   maps: a transposed copy S^T [C][nx][N] (k_transpose_maps), so one
//         column's maps are N contiguous elements; each warp brings its own
//         columns for the next coil into a per-warp double buffer with a 1D
//         bulk copy completed on a per-warp mbarrier.
//   p, q: row-major images, staged once per tile through shared memory
//         (coalesced global access, transposed to [column][row]).
// ---------------------------------------------------------------------------
template <class C, class St>
struct WSmem {
  float2* tw;   // stage twiddle tables (C::TWN)
  float2* buf0;  // W * CP
  float2* buf1;
  double* red;   // 32
  short* map;    // N
  typename St::T* sbuf;  // [warps][2][32 / T * N]
  uint64_t* bar;         // [warps][2]
};

template <class C, class St>
__host__ __device__ constexpr size_t wcol_smem_bytes() {
  constexpr int warps = C::THREADS / 32;
  constexpr size_t per_slot = (size_t)(32 / C::T) * C::N * sizeof(typename St::T);
  size_t b = sizeof(float2) * ((size_t)C::TWN + 2 * (size_t)C::W * C::CP) + 32 * sizeof(double) +
             sizeof(short) * (size_t)C::N;
  b = (b + 15) & ~(size_t)15;
  b += (size_t)warps * 2 * per_slot;
  b += (size_t)warps * 2 * sizeof(uint64_t);
  return b;
}

template <class C, class St>
__device__ __forceinline__ WSmem<C, St> wcol_smem(unsigned char* base) {
  WSmem<C, St> s;
  s.tw = reinterpret_cast<float2*>(base);
  s.buf0 = s.tw + C::TWN;
  s.buf1 = s.buf0 + C::W * C::CP;
  s.red = reinterpret_cast<double*>(s.buf1 + C::W * C::CP);
  s.map = reinterpret_cast<short*>(s.red + 32);
  size_t off = sizeof(float2) * ((size_t)C::TWN + 2 * (size_t)C::W * C::CP) + 32 * sizeof(double) +
               sizeof(short) * (size_t)C::N;
  off = (off + 15) & ~(size_t)15;
  s.sbuf = reinterpret_cast<typename St::T*>(base + off);
  constexpr int warps = C::THREADS / 32;
  off += (size_t)warps * 2 * (size_t)(32 / C::T) * C::N * sizeof(typename St::T);
  s.bar = reinterpret_cast<uint64_t*>(base + off);
  return s;
}

// Stage twiddle tables from the full table tw[m] = exp(-2 pi i m / N):
// table s holds tw[r k Q_s] at (k - 1) P_s + r.
template <class C, class Rad, int s>
__device__ __forceinline__ void wcol_fill_stage(float2* dst, const float2* tw) {
  if constexpr (s < Rad::S - 1) {
    constexpr int R = Rad::radix(s), P = Rad::P(s), Q = Rad::Q(s);
    for (int i = threadIdx.x; i < (R - 1) * P; i += C::THREADS) {
      const int k = i / P + 1, r = i - (k - 1) * P;
      dst[C::twoff(s) + i] = tw[r * k * Q];
    }
    wcol_fill_stage<C, Rad, s + 1>(dst, tw);
  }
}

template <class C>
struct WColRad;
template <int T, int W, class Rad, class Lay>
struct WColRad<WCol<T, W, Rad, Lay>> {
  using type = Rad;
};

// Block start: stage tables and the per-warp barriers (thread 0 initialises
// them; the caller's next __syncthreads publishes both).
template <class C, class St>
__device__ __forceinline__ void wcol_setup(const WSmem<C, St>& s, const float2* tw) {
  wcol_fill_stage<C, typename WColRad<C>::type, 0>(s.tw, tw);
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2 * (C::THREADS / 32); ++i) mbar_init(s.bar + i, 1);
    mbar_fence_init();
  }
}

// One tile: `fill` counts the map copies this block has issued before (the
// same number in every thread); the tile issues a.coils more.  Returns this
// thread's share of Re<p, q> (CG) as normal_tile does.
template <class C, class St, bool CG>
__device__ __forceinline__ float normal_tile_warp(const NormalTile& a, const WSmem<C, St>& s, unsigned keep,
                                                  unsigned fill, int* err, const int* lines = nullptr, int L = 0) {
  constexpr int N = C::N, W = C::W, T = C::T, CW = 32 / T, CP = C::CP;
  using E = typename St::T;
  const C col;
  const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
  const int x0 = a.tile * W;
  const int xw = x0 + warp * CW;  // first column of this warp
  int ncw = a.nx - xw;
  ncw = ncw < 0 ? 0 : (ncw > CW ? CW : ncw);
  const bool xin = x0 + col.c < a.nx;
  const E* ST = static_cast<const E*>(a.S);
  E* sb0 = s.sbuf + (size_t)warp * 2 * CW * N;
  uint64_t* bar = s.bar + 2 * warp;
  const unsigned bytes = (unsigned)(ncw * N * (int)sizeof(E));

  // lane 0: maps of coil `coil` for this warp's columns into slot i & 1
  auto issue = [&](unsigned i, int coil) {
    uint64_t* b = bar + (i & 1);
    if (ncw > 0) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(b, bytes);
      bulk_load(sb0 + (i & 1) * CW * N, ST + ((size_t)coil * a.nx + xw) * N, bytes, b);
    } else {
      mbar_arrive(b);  // keeps the barrier's phases in step with `fill`
    }
  };
  if (lane == 0) issue(fill, 0);

  // p (CG: p = r + beta p_prev, written back) staged as [column][row].  A
  // thread's loads are all issued before the first is used, so their L2
  // latencies overlap instead of adding up.
  constexpr int PER = N * W / C::THREADS;
  static_assert(PER * C::THREADS == N * W, "whole staging rounds");
  {
    float2 pv[PER], rv[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int i = (int)threadIdx.x + u * C::THREADS;
      const int row = i / W, xx = x0 + (i - row * W);
      pv[u] = make_float2(0.f, 0.f);
      rv[u] = make_float2(0.f, 0.f);
      if (xx < a.nx) {
        const size_t idx = (size_t)row * a.nx + xx;
        if (CG) {
          pv[u] = __ldcg(a.p_src + idx);
          if (a.p_update) rv[u] = __ldcg(a.r + idx);
        } else {
          pv[u] = __ldg(a.x + idx);
        }
      }
    }
    if (lines) {  // the frame's line map (and this lane's mask), built while the loads are in flight
      build_linemap<N, C::THREADS>(s.map, lines, L, err);
      keep = sampled_bits<C>(s.map);
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int i = (int)threadIdx.x + u * C::THREADS;
      const int row = i / W, cc = i - row * W, xx = x0 + cc;
      float2 v = pv[u];
      if (xx < a.nx) {
        if (CG) {
          if (a.p_update) {
            v = pfma(splat(a.beta), v, rv[u]);
            __stcg(a.p_dst + (size_t)row * a.nx + xx, v);
          }
        } else {
          v = negate_if(v, a.centred && ((row + xx) & 1));
        }
      }
      s.buf0[cc * CP + row] = v;
    }
  }
  __syncthreads();
  float2 p[C::J0][C::R0], q[C::J0][C::R0], ql[C::J0][C::R0];  // q: compensated coil sum
#pragma unroll
  for (int j = 0; j < C::J0; ++j)
#pragma unroll
    for (int n = 0; n < C::R0; ++n) {
      p[j][n] = col.ok0(j) ? s.buf0[col.c * CP + col.xrow(j, n)] : make_float2(0.f, 0.f);
      q[j][n] = make_float2(0.f, 0.f);
      ql[j][n] = make_float2(0.f, 0.f);
    }

  float2* bufs[2] = {s.buf0, s.buf1};
  const typename C::Tw0 w0 = col.load_tw0(s.tw);
  const int cw = col.c - warp * CW;  // column within the warp
#pragma unroll 1
  for (int c = 0; c < a.coils; ++c) {
    const unsigned i = fill + (unsigned)c;
    __syncwarp();  // every lane is done with slot (i + 1) & 1 and with its p reads
    if (lane == 0 && c + 1 < a.coils) issue(i + 1, c + 1);
    if (!mbar_wait(bar + (i & 1), (i >> 1) & 1u)) atomicOr(err, ERR_TIMEOUT);
    const E* sc = sb0 + (i & 1) * CW * N + cw * N;
    float2 xr[C::J0][C::R0];
    float2 kr[C::JL][C::RL];
#pragma unroll
    for (int j = 0; j < C::J0; ++j)
#pragma unroll
      for (int n = 0; n < C::R0; ++n) {
        const float2 sv = col.ok0(j) ? St::lds(sc, col.xrow(j, n)) : make_float2(0.f, 0.f);
        xr[j][n] = cmul(sv, p[j][n]);
      }
    col.fwd(xr, kr, bufs, s.tw, w0);
#pragma unroll
    for (int j = 0; j < C::JL; ++j)
#pragma unroll
      for (int m = 0; m < C::RL; ++m)
        if (!((keep >> (j * C::RL + m)) & 1u)) kr[j][m] = make_float2(0.f, 0.f);
    col.inv(kr, xr, bufs, s.tw, w0);
#pragma unroll
    for (int j = 0; j < C::J0; ++j)
#pragma unroll
      for (int n = 0; n < C::R0; ++n) {
        const float2 sv = col.ok0(j) ? St::lds(sc, col.xrow(j, n)) : make_float2(0.f, 0.f);
        csum_fma_conj(q[j][n], ql[j][n], sv, xr[j][n]);
      }
  }

  // q staged as [column][row], then stored row-major
  const float invN = 1.0f / (float)N;
  float part = 0.f;
  __syncwarp();
#pragma unroll
  for (int j = 0; j < C::J0; ++j)
#pragma unroll
    for (int n = 0; n < C::R0; ++n) {
      if (!col.ok0(j)) continue;
      float2 qv = cscale(csum_value(q[j][n], ql[j][n]), invN);
      if (CG) {
        qv = make_float2(fmaf(a.lambda, p[j][n].x, qv.x), fmaf(a.lambda, p[j][n].y, qv.y));
        if (a.lambda_t != 0.f && xin) qv = cadd(qv, temporal_term(a, (size_t)col.xrow(j, n) * a.nx + x0 + col.c, p[j][n]));
      }
      s.buf0[col.c * CP + col.xrow(j, n)] = qv;
      if (CG && xin) part = fmaf(p[j][n].x, qv.x, fmaf(p[j][n].y, qv.y, part));
    }
  __syncthreads();
  for (int i = threadIdx.x; i < N * W; i += C::THREADS) {
    const int row = i / W, cc = i - row * W, xx = x0 + cc;
    if (xx < a.nx) {
      const size_t idx = (size_t)row * a.nx + xx;
      if (CG)
        __stcg(a.q + idx, s.buf0[cc * CP + row]);
      else
        a.out[idx] = negate_if(s.buf0[cc * CP + row], a.centred && ((row + xx) & 1));
    }
  }
  return part;
}

// S [C][N][nx] -> S^T [C][nx][N] (storage type kept), 32 x 32 tiles.
template <class E>
__global__ void __launch_bounds__(256) k_transpose_maps(const E* __restrict__ S, E* __restrict__ ST, int N, int nx) {
  __shared__ E tile[32][33];
  const int c = blockIdx.z;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * 32;
  const E* src = S + (size_t)c * N * nx;
  E* dst = ST + (size_t)c * N * nx;
  for (int yy = threadIdx.y; yy < 32; yy += 8) {
    const int y = y0 + yy, x = x0 + threadIdx.x;
    if (y < N && x < nx) tile[yy][threadIdx.x] = src[(size_t)y * nx + x];
  }
  __syncthreads();
  for (int xx = threadIdx.y; xx < 32; xx += 8) {
    const int x = x0 + xx, y = y0 + threadIdx.x;
    if (y < N && x < nx) dst[(size_t)x * N + y] = tile[threadIdx.x][xx];
  }
}

template <class C>
__device__ __forceinline__ unsigned sampled_bits(const ColSmem& s) {
  return sampled_bits<C>(s.map);
}

template <class St>
struct NormalArgs {
  const float2* x;             // CG=false input
  float2* out;                 // CG=false output
  const float2* p_src;         // CG=true: previous search direction (or the current one if !p_update)
  float2* p_dst;               // CG=true: new search direction (written when p_update)
  const float2* r;             // CG=true
  float2* q;                   // CG=true output
  const typename St::T* S;
  const int* lines;
  const float2* tw;
  int nx, coils, L, tiles, p_update;
  int centred;                 // CG=false: centred k-space (see NormalTile)
  float lambda;                // CG=true: Tikhonov weight
  int* err;
  CgState cg;
};

// shared memory of k_normal for configuration C (either engine)
template <class C, class St>
__host__ __device__ constexpr size_t normal_smem_bytes() {
  if constexpr (is_wcol<C>::value)
    return wcol_smem_bytes<C, St>();
  else
    return col_smem_bytes_c<C>();
}

template <int N, int V, class St, bool CG, int TH = NormCfg<N, V>::C::THREADS, int MINB = NormCfg<N, V>::MINB>
__global__ void __launch_bounds__(TH, MINB) k_normal(NormalArgs<St> a) {
  using C = typename NormCfg<N, V>::C;
  const int f = blockIdx.y;
  if (CG && a.cg.active[f] == 0) return;  // uniform per block
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const size_t img = (size_t)N * a.nx;
  NormalTile t;
  t.x = a.x + f * img;
  t.out = a.out + f * img;
  t.p_src = a.p_src + f * img;
  t.p_dst = a.p_dst + f * img;
  t.r = a.r + f * img;
  t.q = a.q + f * img;
  t.S = a.S;
  t.nx = a.nx;
  t.coils = a.coils;
  t.tile = blockIdx.x;
  t.p_update = a.p_update;
  t.centred = CG ? 0 : a.centred;
  t.lambda = CG ? a.lambda : 0.f;
  t.lambda_t = 0.f;  // frames are coupled only in the persistent kernel
  t.beta = (CG && a.p_update) ? (float)__ldg(a.cg.beta + f) : 0.f;
  float part;
  double* red;
  if constexpr (is_wcol<C>::value) {  // a.S holds the transposed maps
    const WSmem<C, St> s = wcol_smem<C, St>(smem_raw);
    wcol_setup<C, St>(s, a.tw);
    build_linemap<N, C::THREADS>(s.map, a.lines + (size_t)f * a.L, a.L, a.err);
    part = normal_tile_warp<C, St, CG>(t, s, sampled_bits<C>(s.map), 0u, a.err);
    red = s.red;
  } else {
    const ColSmem s = col_smem_c<C>(smem_raw);
    load_tw_and_linemap<N, C::THREADS>(s, a.tw, a.lines + (size_t)f * a.L, a.L, a.err);
    part = normal_tile<C, St, CG>(t, s, sampled_bits<C>(s));
    red = s.red;
  }
  if (CG) {
    const double tot = block_sum<C::THREADS>((double)part, red);
    const CgState& g = a.cg;
    double* slot = g.part + (size_t)f * g.part_stride + blockIdx.x;
    if (publish_and_arrive(tot, slot, g.counter + f, (unsigned)a.tiles)) {
      const double pq = ordered_sum(g.part + (size_t)f * g.part_stride, a.tiles);
      g.counter[f] = 0u;
      if (pq > 0.0) {
        g.alpha[f] = g.rho[f] / pq;
      } else {  // breakdown (zero, negative or NaN curvature): freeze the frame
        g.active[f] = 0;
        g.outcome[f] = CG_BREAKDOWN;
        atomicSub(g.live, 1);
      }
    }
  }
}

}  // namespace sense

// Column passes of E and E^H as persistent kernels whose per-coil tiles
// arrive by TMA.
//
// A block loops over (frame, column tile) items, blockIdx.x, + gridDim.x, ...
// Per coil it needs the [N][W] tile of the maps S_c and (E^H) the [L][W]
// tile of the row-transformed k-space of (frame, coil); both come from 2D
// tiled bulk copies (cp.async.bulk.tensor) into one of two shared-memory
// slots, completing on that slot's mbarrier.  The copy for the next coil --
// of this item, or the first coil of the block's next item -- is issued at
// the top of each coil, so its latency hides behind a whole coil's transform
// and no block ever waits on an empty pipe except at its first item.
//
// Fill i of a block goes to slot i & 1 and completes phase (i >> 1) & 1 of
// that slot's barrier.  Each coil starts with every thread waiting for its
// fill and a block barrier that ANDs the outcomes; only then does thread 0
// issue the next fill, into the slot the previous coil read, which every
// thread has finished with by then.  Waits are bounded: a fill that never
// lands sets ERR_TIMEOUT, waits once more for the copy (bounded), and the
// whole block skips the item's stores, leaving those outputs as they were.
//
// Tensor maps are kernel parameters (__grid_constant__), encoded on the host
// for each call: S as [C*N] rows of nx elements (box W x NB rows, two boxes
// when N > 256), the intermediate as [F*C*L] rows of nx complex values (box
// W x LB rows, two boxes when L > 256).  The x coordinate of every copy is
// tile * W, W = 8: a multiple of 16 bytes for both storages.
#pragma once
#include <cuda.h>

#include "kernels.cuh"

namespace sense {

// The length's transform on 8-column tiles (the x coordinate of every copy a
// multiple of 16 bytes); lengths whose tile would not fill whole warps keep
// the register-staged column kernels.
template <int N>
struct ColTma;
// every S slot and the second S box start 128 bytes after an aligned one
template <int N, class St>
constexpr bool stiles_aligned() {
  return ((size_t)N * 8 * sizeof(typename St::T)) % 128 == 0 && ((size_t)(N / 2) * 8 * sizeof(typename St::T)) % 128 == 0;
}

template <int N>
struct ColTma {
  using Base = typename Cfg<N>::C;
  static constexpr int W = 8;
  using C = Col<Base::T, W, typename Base::Radix>;
  static constexpr bool ok = (Base::T * W) % 32 == 0;
  static constexpr int MINB = C::THREADS <= 384 ? 2 : 1;  // two blocks per SM: register cap 128 (256 threads) to 85 (384)
  static constexpr int NB = N <= 256 ? N : N / 2;         // rows per S box
  static_assert(N <= 256 || N % 2 == 0, "two S boxes need an even length");
};

// Rows per box of the intermediate (one box for up to 256 lines, two above)
// and the rows a slot holds.  A tensor copy's shared-memory destination must
// be 128-byte aligned: a box row is W = 8 complex values (64 bytes), so boxes
// and slots hold an even number of rows (a box may read one row past the
// frame's lines, which is never used).
__host__ __device__ constexpr int kbox_rows(int L) { return L <= 256 ? (L + 1) & ~1 : (((L + 1) / 2) + 1) & ~1; }
__host__ __device__ constexpr int kslot_rows(int L) { return L <= 256 ? kbox_rows(L) : 2 * kbox_rows(L); }
static_assert(kbox_rows(21) == 22 && kbox_rows(256) == 256 && kbox_rows(301) == 152 && kbox_rows(384) == 192,
              "box rows");

// shared memory: twiddles, two exchange buffers, FP64 scratch, line map,
// two S slots, two k-space slots (E^H only), two barriers
template <int N, class St>
__host__ __device__ constexpr size_t coltma_smem_bytes(int L, bool with_k) {
  using C = typename ColTma<N>::C;
  size_t b = col_smem_bytes_c<C>();
  b = (b + 127) & ~(size_t)127;
  b += 2 * (size_t)N * C::W * sizeof(typename St::T);
  b = (b + 127) & ~(size_t)127;
  if (with_k) b += 2 * (size_t)kslot_rows(L) * C::W * sizeof(float2);
  b = (b + 15) & ~(size_t)15;
  return b + 2 * sizeof(uint64_t);
}

template <int N, class St>
struct ColTmaSmem {
  static_assert(stiles_aligned<N, St>(), "S slots must stay 128-byte aligned");
  ColSmem s;
  typename St::T* sb[2];
  float2* kb[2];
  uint64_t* bar;
  __device__ __forceinline__ ColTmaSmem(unsigned char* base, int L, bool with_k) {
    using C = typename ColTma<N>::C;
    s = col_smem_c<C>(base);
    size_t off = (col_smem_bytes_c<C>() + 127) & ~(size_t)127;
    sb[0] = reinterpret_cast<typename St::T*>(base + off);
    sb[1] = sb[0] + (size_t)N * C::W;
    off += 2 * (size_t)N * C::W * sizeof(typename St::T);
    off = (off + 127) & ~(size_t)127;
    kb[0] = reinterpret_cast<float2*>(base + off);
    kb[1] = kb[0] + (size_t)kslot_rows(L) * C::W;
    if (with_k) off += 2 * (size_t)kslot_rows(L) * C::W * sizeof(float2);
    off = (off + 15) & ~(size_t)15;
    bar = reinterpret_cast<uint64_t*>(base + off);
  }
};

// thread 0: fill slot i & 1 with coil c of item (f, tile)
template <int N, class St, bool WITH_S, bool WITH_K>
__device__ __forceinline__ void coltma_issue(const ColTmaSmem<N, St>& m, const CUtensorMap* tmS,
                                             const CUtensorMap* tmK, unsigned i, int f, int tile, int c,
                                             int coils, int L) {
  using T = ColTma<N>;
  constexpr int W = T::W;
  const int slot = (int)(i & 1u);
  uint64_t* b = m.bar + slot;
  unsigned bytes = 0;
  if (WITH_S) bytes += (unsigned)(N * W * sizeof(typename St::T));
  const int LB = kbox_rows(L);
  if (WITH_K) bytes += (unsigned)((L <= 256 ? 1 : 2) * LB * W * sizeof(float2));
  fence_proxy_async_smem();
  mbar_arrive_expect_tx(b, bytes);
  if (WITH_S) {
    typename St::T* dst = slot ? m.sb[1] : m.sb[0];
    tma_load_2d(dst, tmS, tile * W, c * N, b);
    if (N > 256) tma_load_2d(dst + T::NB * W, tmS, tile * W, c * N + T::NB, b);
  }
  if (WITH_K) {
    float2* dst = slot ? m.kb[1] : m.kb[0];
    const int row = (f * coils + c) * L;
    tma_load_2d(dst, tmK, tile * W, row, b);
    if (L > 256) tma_load_2d(dst + LB * W, tmK, tile * W, row + LB, b);
  }
}

// Wait for fill i; false (and ERR_TIMEOUT raised) if it did not land in time.
__device__ __forceinline__ bool coltma_wait(uint64_t* bar, unsigned i, int* err) {
  uint64_t* b = bar + (i & 1u);
  const unsigned parity = (i >> 1) & 1u;
  if (mbar_wait(b, parity)) return true;
  if (threadIdx.x == 0) atomicOr(err, ERR_TIMEOUT);
  mbar_wait(b, parity);  // let the copy land before the slot is reused
  return false;
}

// ---------------------------------------------------------------------------
// E^H column pass.  MODE 0: x = sum_c conj(S_c) F_y^H(...); MODE 1: the same
// written as the CG start (r = p = b, x = 0, rho0); MODE 2: root sum of squares.
// ---------------------------------------------------------------------------
template <int N, class St, int MODE, int TH = ColTma<N>::C::THREADS>
__global__ void __launch_bounds__(TH, ColTma<N>::MINB)
    k_adj_col_tma(const __grid_constant__ CUtensorMap tmK, const __grid_constant__ CUtensorMap tmS,
                  AdjColArgs<St> a, int frames) {
  using C = typename ColTma<N>::C;
  constexpr int W = C::W;
  constexpr bool WITH_S = MODE != 2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  if (smem_addr(smem_raw) & 127u) {  // tensor copies need 128-byte aligned destinations
    if (threadIdx.x == 0) atomicOr(a.err, ERR_TIMEOUT);
    return;
  }
  const ColTmaSmem<N, St> m(smem_raw, a.L, true);
  const ColSmem& s = m.s;
  const C col;
  const int items = a.tiles * frames;
  const size_t img = (size_t)N * a.nx;
  for (int i = threadIdx.x; i < N; i += C::THREADS) s.tw[i] = a.tw[i];
  if (threadIdx.x == 0) {
    mbar_init(m.bar, 1);
    mbar_init(m.bar + 1, 1);
    mbar_fence_init();
  }
  __syncthreads();
  int item = blockIdx.x;
  if (threadIdx.x == 0 && item < items)
    coltma_issue<N, St, WITH_S, true>(m, &tmS, &tmK, 0u, item / a.tiles, item % a.tiles, 0, a.coils, a.L);
  // register twiddles (loaded once, used by every coil) where the register cap leaves room
  constexpr bool REG_TW = MODE == 2 || 65536 / (C::THREADS * ColTma<N>::MINB) >= 160;
  typename C::Tw0 w0;
  if constexpr (REG_TW) w0 = col.load_tw0(s.tw);
  unsigned fill = 0;  // fills consumed so far
  int mapped_f = -1;
  const float scale = rsqrtf((float)N);
  for (; item < items; item += gridDim.x) {
    const int f = item / a.tiles, tile = item - f * a.tiles;
    const int x = tile * W + col.c;
    const bool xin = x < a.nx;
    if (f != mapped_f) {  // line map of this frame
      __syncthreads();    // every thread is past the previous item's reads of the map
      for (int i = threadIdx.x; i < N; i += C::THREADS) s.map[i] = -1;
      __syncthreads();
      const int* ln = a.lines + (size_t)f * a.L;
      for (int l = threadIdx.x; l < a.L; l += C::THREADS) {
        const int v = __ldg(ln + l);
        const bool good = v >= 0 && v < N && (l == 0 || __ldg(ln + l - 1) < v);
        if (good)
          s.map[v] = (short)l;
        else
          atomicOr(a.err, ERR_LINES);
      }
      __syncthreads();
      mapped_f = f;
    }
    float2 acc[C::J0][C::R0], accl[C::J0][C::R0];
    float accr[C::J0][C::R0];
#pragma unroll
    for (int j = 0; j < C::J0; ++j)
#pragma unroll
      for (int n = 0; n < C::R0; ++n) {
        acc[j][n] = make_float2(0.f, 0.f);
        accl[j][n] = make_float2(0.f, 0.f);
        accr[j][n] = 0.f;
      }
    bool landed = true;  // the same in every thread
#pragma unroll 1
    for (int c = 0; c < a.coils; ++c, ++fill) {
      // every thread has this coil's tiles and is done with the previous coil's slot
      landed = __syncthreads_and(coltma_wait(m.bar, fill, a.err)) && landed;
      if (threadIdx.x == 0) {
        if (c + 1 < a.coils) {
          coltma_issue<N, St, WITH_S, true>(m, &tmS, &tmK, fill + 1, f, tile, c + 1, a.coils, a.L);
        } else if (item + (int)gridDim.x < items) {
          const int nx_item = item + gridDim.x;
          coltma_issue<N, St, WITH_S, true>(m, &tmS, &tmK, fill + 1, nx_item / a.tiles, nx_item % a.tiles, 0,
                                            a.coils, a.L);
        }
      }
      const float2* kb = (fill & 1u) ? m.kb[1] : m.kb[0];
      float2 kr[C::JL][C::RL];
      float2 xr[C::J0][C::R0];
#pragma unroll
      for (int j = 0; j < C::JL; ++j)
#pragma unroll
        for (int m2 = 0; m2 < C::RL; ++m2) {
          const int row = col.krow(j, m2);
          const int l = col.okL(j) ? (int)s.map[row] : -1;
          float2 v = l >= 0 ? kb[l * W + col.c] : make_float2(0.f, 0.f);
          kr[j][m2] = negate_if(v, a.centred && (row & 1));
        }
      const BufPair<C> bp(s.buf0, s.buf1, c);
      if constexpr (REG_TW)
        col.inv(kr, xr, bp.b, s.tw, w0);
      else
        col.inv(kr, xr, bp.b, s.tw);
      const typename St::T* sb = (fill & 1u) ? m.sb[1] : m.sb[0];
#pragma unroll
      for (int j = 0; j < C::J0; ++j)
#pragma unroll
        for (int n = 0; n < C::R0; ++n) {
          if (MODE == 2) {
            accr[j][n] = fmaf(xr[j][n].x, xr[j][n].x, fmaf(xr[j][n].y, xr[j][n].y, accr[j][n]));
          } else {
            const float2 sv = col.ok0(j) ? St::lds(sb, col.xrow(j, n) * W + col.c) : make_float2(0.f, 0.f);
            csum_fma_conj(acc[j][n], accl[j][n], sv, xr[j][n]);
          }
        }
    }
    float part = 0.f;
    if (landed) {
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
    }
    if (MODE == 1) {
      const double tot = block_sum<C::THREADS>((double)part, s.red);
      const CgState& g = a.cg;
      double* slot = g.part + (size_t)f * g.part_stride + tile;
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
}

// ---------------------------------------------------------------------------
// E column pass: per coil S_c . x (x tile in registers for the whole item),
// F_y, sampled rows stored to the intermediate [F][C][L][nx].
// ---------------------------------------------------------------------------
template <int N, class St, int TH = ColTma<N>::C::THREADS>
__global__ void __launch_bounds__(TH, ColTma<N>::MINB)
    k_fwd_col_tma(const __grid_constant__ CUtensorMap tmS, FwdColArgs<St> a, int tiles, int frames) {
  using C = typename ColTma<N>::C;
  constexpr int W = C::W;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  if (smem_addr(smem_raw) & 127u) {  // tensor copies need 128-byte aligned destinations
    if (threadIdx.x == 0) atomicOr(a.err, ERR_TIMEOUT);
    return;
  }
  const ColTmaSmem<N, St> m(smem_raw, a.L, false);
  const ColSmem& s = m.s;
  const C col;
  const int items = tiles * frames;
  const size_t img = (size_t)N * a.nx;
  for (int i = threadIdx.x; i < N; i += C::THREADS) s.tw[i] = a.tw[i];
  if (threadIdx.x == 0) {
    mbar_init(m.bar, 1);
    mbar_init(m.bar + 1, 1);
    mbar_fence_init();
  }
  __syncthreads();
  int item = blockIdx.x;
  if (threadIdx.x == 0 && item < items)
    coltma_issue<N, St, true, false>(m, &tmS, nullptr, 0u, item / tiles, item % tiles, 0, a.coils, a.L);
  unsigned fill = 0;
  int mapped_f = -1;
  const float scale = rsqrtf((float)N);
  for (; item < items; item += gridDim.x) {
    const int f = item / tiles, tile = item - f * tiles;
    const int x = tile * W + col.c;
    const bool xin = x < a.nx;
    if (f != mapped_f) {  // line map of this frame
      __syncthreads();    // every thread is past the previous item's stores, which read the map
      for (int i = threadIdx.x; i < N; i += C::THREADS) s.map[i] = -1;
      __syncthreads();
      const int* ln = a.lines + (size_t)f * a.L;
      for (int l = threadIdx.x; l < a.L; l += C::THREADS) {
        const int v = __ldg(ln + l);
        const bool good = v >= 0 && v < N && (l == 0 || __ldg(ln + l - 1) < v);
        if (good)
          s.map[v] = (short)l;
        else
          atomicOr(a.err, ERR_LINES);
      }
      __syncthreads();
      mapped_f = f;
    }
    float2 xv[C::J0][C::R0];
#pragma unroll
    for (int j = 0; j < C::J0; ++j)
#pragma unroll
      for (int n = 0; n < C::R0; ++n)
        xv[j][n] = (col.ok0(j) && xin) ? negate_if(__ldg(a.x + f * img + (size_t)col.xrow(j, n) * a.nx + x),
                                                   a.centred && ((col.xrow(j, n) + x) & 1))
                                        : make_float2(0.f, 0.f);
#pragma unroll 1
    for (int c = 0; c < a.coils; ++c, ++fill) {
      // every thread has this coil's maps and is done with the previous coil's slot
      const bool landed = __syncthreads_and(coltma_wait(m.bar, fill, a.err));
      if (threadIdx.x == 0) {
        if (c + 1 < a.coils) {
          coltma_issue<N, St, true, false>(m, &tmS, nullptr, fill + 1, f, tile, c + 1, a.coils, a.L);
        } else if (item + (int)gridDim.x < items) {
          const int nx_item = item + gridDim.x;
          coltma_issue<N, St, true, false>(m, &tmS, nullptr, fill + 1, nx_item / tiles, nx_item % tiles, 0,
                                           a.coils, a.L);
        }
      }
      const typename St::T* sb = (fill & 1u) ? m.sb[1] : m.sb[0];
      float2 xr[C::J0][C::R0];
      float2 kr[C::JL][C::RL];
#pragma unroll
      for (int j = 0; j < C::J0; ++j)
#pragma unroll
        for (int n = 0; n < C::R0; ++n) {
          const float2 sv = col.ok0(j) ? St::lds(sb, col.xrow(j, n) * W + col.c) : make_float2(0.f, 0.f);
          xr[j][n] = cmul(sv, xv[j][n]);
        }
      const BufPair<C> bp(s.buf0, s.buf1, c);
      col.fwd(xr, kr, bp.b, s.tw);
      if (!landed) continue;
      float2* dst = a.tmp + ((size_t)f * a.coils + c) * a.L * a.nx;
#pragma unroll
      for (int j = 0; j < C::JL; ++j)
#pragma unroll
        for (int m2 = 0; m2 < C::RL; ++m2) {
          if (col.okL(j) && xin) {
            const int l = s.map[col.krow(j, m2)];
            if (l >= 0)
              dst[(size_t)l * a.nx + x] = negate_if(cscale(kr[j][m2], scale), a.centred && (col.krow(j, m2) & 1));
          }
        }
    }
  }
}

}  // namespace sense

// Both passes of E^H (adjoint, CG start, root-sum-of-squares) or of E in one
// persistent launch, with the row-transformed intermediate kept in L2.
//
// The two-pass operators run the x-direction (row) transforms of the
// sampled k-space rows and the y-direction (column) transforms with the maps
// as two launches: the second starts only when the first has finished, and
// for problems larger than L2 the whole compacted intermediate travels to
// HBM and back.  Here one launch runs both kinds of work item:
//   first pass  (E^H: a tile of 8 rows of one frame; E: a tile of 8 columns)
//   second pass (E^H: a tile of 8 columns;           E: a tile of 8 rows)
// handed out by one ticket counter in a frame-staggered order: stage s holds
// the first-pass tiles of frame s, then the second-pass tiles of frame s - 1.
// A second-pass item of frame f waits (thread 0, bounded) until every
// first-pass tile of f has stored its rows; those have smaller tickets, taken
// by blocks that are already running (the grid is one wave of resident
// blocks), so every wait ends.  At any moment only the intermediate of about
// two frames is live, so it stays in L2; and one frame's memory-heavy row
// tiles overlap another frame's transform-heavy column tiles.
//
// Square images only (the row and column transforms then share one engine
// configuration, block size and twiddle table).  Column tiles stage each
// coil's map tile (and, for E^H, its k-space tile) by TMA as the persistent
// column passes do (colpass.cuh), one coil ahead within an item.  Row tiles
// move rows through shared memory with coalesced loads and stores.
//
// Ordering: a first-pass tile's threads store, fence (__threadfence) and
// meet at a barrier before thread 0 counts the tile; the waiting thread
// acquires the count, and (E^H) orders the tensor copies that follow after
// it (fence.proxy.async.global); E's row tiles read the intermediate through
// L2 (ld.global.cg).
#pragma once
#include <type_traits>

#include "colpass.cuh"
#include "persistent.cuh"

namespace sense {

struct FusedSched {
  unsigned* ticket;  // zeroed before the launch
  int* done;         // [frames] first-pass items stored, zeroed before the launch
  int frames;
  int first_tiles;   // first-pass items per frame
  int second_tiles;  // second-pass items per frame
  int lag;           // second-pass items of frame f follow the first-pass items of frame f + lag
};

// Row items move kFusedRowTiles tiles of 8 rows each (fewer, longer items).
constexpr int kFusedRowTiles = 4;
// Second-pass items of frame f come after the first-pass items of frame f + kFusedLag.
constexpr int kFusedLag = 3;

// Shared memory of the fused kernels: twiddles, one exchange region used by
// either pass (column engine: two N x 8 buffers; row engine: the 8-row tile
// of pitch N + 2 and one N x 8 buffer), FP64 scratch, line map, two map
// slots, two k-space slots (E^H), two barriers.
template <int N, class St>
__host__ __device__ constexpr size_t fused_smem_bytes(int L, bool with_k) {
  size_t b = sizeof(float2) * (size_t)N;                     // twiddles
  b += sizeof(float2) * 8 * (2 * (size_t)N + 2);             // exchange region
  b += 32 * sizeof(double) + sizeof(short) * (size_t)N;      // red, map
  b = (b + 127) & ~(size_t)127;
  b += 2 * (size_t)N * 8 * sizeof(typename St::T);           // map slots
  b = (b + 127) & ~(size_t)127;
  if (with_k) b += 2 * (size_t)kslot_rows(L) * 8 * sizeof(float2);
  b = (b + 15) & ~(size_t)15;
  return b + 2 * sizeof(uint64_t);
}

template <int N, class St>
struct FusedSmem {
  ColTmaSmem<N, St> m;  // column-pass view (its buffers point into the exchange region)
  float2* tile;         // row pass: 8 rows of pitch N + 2
  float2* rbuf;         // row pass: second exchange buffer, N x 8
  __device__ __forceinline__ FusedSmem(unsigned char* base, int L, bool with_k) : m(base, 0, false) {
    float2* tw = reinterpret_cast<float2*>(base);
    float2* x = tw + N;
    m.s.tw = tw;
    m.s.buf0 = x;
    m.s.buf1 = x + 8 * (size_t)N;
    tile = x;
    rbuf = x + 8 * ((size_t)N + 2);
    m.s.red = reinterpret_cast<double*>(x + 8 * (2 * (size_t)N + 2));
    m.s.map = reinterpret_cast<short*>(m.s.red + 32);
    size_t off = sizeof(float2) * ((size_t)N + 8 * (2 * (size_t)N + 2)) + 32 * sizeof(double) + sizeof(short) * N;
    off = (off + 127) & ~(size_t)127;
    m.sb[0] = reinterpret_cast<typename St::T*>(base + off);
    m.sb[1] = m.sb[0] + (size_t)N * 8;
    off += 2 * (size_t)N * 8 * sizeof(typename St::T);
    off = (off + 127) & ~(size_t)127;
    m.kb[0] = reinterpret_cast<float2*>(base + off);
    m.kb[1] = m.kb[0] + (size_t)kslot_rows(L) * 8;
    if (with_k) off += 2 * (size_t)kslot_rows(L) * 8 * sizeof(float2);
    off = (off + 15) & ~(size_t)15;
    m.bar = reinterpret_cast<uint64_t*>(base + off);
  }
};

// Line map of frame f into s.map (every thread must reach it).
template <int N, int THREADS>
__device__ __forceinline__ void fused_linemap(const ColSmem& s, const int* lines, int L, int f, int* err) {
  __syncthreads();  // every thread is past earlier reads of the map
  for (int i = threadIdx.x; i < N; i += THREADS) s.map[i] = -1;
  __syncthreads();
  const int* ln = lines + (size_t)f * L;
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

// One tile of up to 8 rows of length N, transformed along the row.  DIR = +1:
// inverse (storage in, FP32 out; E^H first pass); DIR = -1: forward (FP32 in
// through L2, storage out; E second pass).  Rows r0 .. r0 + nrows - 1.
template <int N, int DIR, class InSt, class OutSt, class C>
__device__ __forceinline__ void fused_row_tile(const typename InSt::T* in, typename OutSt::T* out, long r0, int nrows,
                                               const float2* tw, float2* tile, float2* rbuf, int centred, float cs) {
  constexpr int P = N + 2;
  constexpr int PER = (8 * N + C::THREADS - 1) / C::THREADS;
  const C col;
  {
    float2 v[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int i = (int)threadIdx.x + k * C::THREADS;
      const int rr = i / N, e = i - rr * N;
      v[k] = make_float2(0.f, 0.f);
      if (i < 8 * N && rr < nrows) {
        if constexpr (DIR > 0)
          v[k] = InSt::ld(in, (size_t)(r0 + rr) * N + e);
        else
          v[k] = __ldcg(reinterpret_cast<const float2*>(in) + (size_t)(r0 + rr) * N + e);
      }
      if (DIR > 0 && centred) v[k] = cscale(v[k], (e & 1) ? -cs : cs);
    }
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int i = (int)threadIdx.x + k * C::THREADS;
      const int rr = i / N, e = i - rr * N;
      if (i < 8 * N) tile[rr * P + e] = v[k];
    }
  }
  __syncthreads();
  const float scale = rsqrtf((float)N);
  float2 xr[C::J0][C::R0];
  float2 kr[C::JL][C::RL];
  float2* row = tile + col.c * P;
  float2* bufs[2] = {tile, rbuf};  // the tile doubles as the first exchange buffer
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
        if (col.okL(j)) row[col.krow(j, m)] = cscale(kr[j][m], scale);
  } else {
#pragma unroll
    for (int j = 0; j < C::JL; ++j)
#pragma unroll
      for (int m = 0; m < C::RL; ++m) kr[j][m] = col.okL(j) ? row[col.krow(j, m)] : make_float2(0.f, 0.f);
    __syncthreads();
    col.inv(kr, xr, bufs, tw);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < C::J0; ++j)
#pragma unroll
      for (int n = 0; n < C::R0; ++n)
        if (col.ok0(j)) row[col.xrow(j, n)] = cscale(xr[j][n], scale);
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int i = (int)threadIdx.x + k * C::THREADS;
    const int rr = i / N, e = i - rr * N;
    if (i < 8 * N && rr < nrows) {
      float2 v = tile[rr * P + e];
      if (DIR < 0 && centred) v = cscale(v, (e & 1) ? -cs : cs);
      if constexpr (DIR > 0)
        reinterpret_cast<float2*>(out)[(size_t)(r0 + rr) * N + e] = v;
      else
        OutSt::st(out, (size_t)(r0 + rr) * N + e, v);
    }
  }
}

// First-pass tile stored: every thread fences its stores, the block meets,
// thread 0 counts the tile for its frame.
__device__ __forceinline__ void fused_count(int* done, int f) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) atomicAdd(done + f, 1);
}

// Thread 0 of a second-pass item: wait for every first-pass tile of frame f.
__device__ __forceinline__ bool fused_wait(const FusedSched& sc, int f, int* err) {
  const bool ok = wait_at_least(sc.done + f, sc.first_tiles);
  if (!ok) atomicOr(err, ERR_TIMEOUT);
  asm volatile("fence.proxy.async.global;" ::: "memory");  // the tensor copies that follow read what was stored
  return ok;
}

// ---------------------------------------------------------------------------
// E^H: first pass = inverse row transforms of the sampled rows of one frame
// (8 of its coils x lines rows per tile) into the intermediate; second pass =
// the column tile of k_adj_col_tma (MODE 0 adjoint, 1 CG start, 2 RSS).
// ---------------------------------------------------------------------------
template <int N, class St, class YSt, int MODE, int TH = ColTma<N>::C::THREADS>
__global__ void __launch_bounds__(TH, ColTma<N>::MINB)
    k_adjoint_fused(const __grid_constant__ CUtensorMap tmK, const __grid_constant__ CUtensorMap tmS,
                    AdjColArgs<St> a, const typename YSt::T* y, float2* tmp_out, FusedSched sc, float cs) {
  // St: storage of S (complex64 for RSS, which reads no maps); YSt: storage of y
  using C = typename ColTma<N>::C;
  constexpr int W = C::W;
  constexpr bool WITH_S = MODE != 2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  if (smem_addr(smem_raw) & 127u) {  // tensor copies need 128-byte aligned destinations
    if (threadIdx.x == 0) atomicOr(a.err, ERR_TIMEOUT);
    return;
  }
  const FusedSmem<N, St> fs(smem_raw, a.L, true);
  const ColTmaSmem<N, St>& m = fs.m;
  const ColSmem& s = m.s;
  __shared__ int s_ticket, s_ok;
  const C col;
  const size_t img = (size_t)N * a.nx;
  const int rows_per_frame = a.coils * a.L;
  const long total = (long)sc.frames * (sc.first_tiles + sc.second_tiles);
  for (int i = threadIdx.x; i < N; i += C::THREADS) s.tw[i] = a.tw[i];
  if (threadIdx.x == 0) {
    mbar_init(m.bar, 1);
    mbar_init(m.bar + 1, 1);
    mbar_fence_init();
  }
  __syncthreads();
  constexpr bool REG_TW = MODE == 2 || 65536 / (C::THREADS * ColTma<N>::MINB) >= 160;
  typename C::Tw0 w0;
  if constexpr (REG_TW) w0 = col.load_tw0(s.tw);
  unsigned fill = 0;
  int mapped_f = -1;
  const float scale = rsqrtf((float)N);
  for (;;) {
    __syncthreads();  // the previous item is done with shared memory and s_*
    if (threadIdx.x == 0) s_ticket = (int)atomicAdd(sc.ticket, 1u);
    __syncthreads();
    const long t = s_ticket;
    if (t >= total) break;
    const StaggeredItem it = staggered_item(t, sc.frames, sc.first_tiles, sc.second_tiles, sc.lag);
    if (!it.second) {  // ---- rows of frame it.unit: kFusedRowTiles tiles of 8 ----
      for (int k = 0; k < kFusedRowTiles; ++k) {
        const int first = (it.piece * kFusedRowTiles + k) * 8;
        if (first >= rows_per_frame) break;
        const int left = rows_per_frame - first;
        if (k > 0) __syncthreads();  // the previous tile's stores have read the shared tile
        fused_row_tile<N, +1, YSt, StC64, C>(y, tmp_out, (long)it.unit * rows_per_frame + first, left < 8 ? left : 8,
                                             s.tw, fs.tile, fs.rbuf, a.centred, cs);
      }
      fused_count(sc.done, it.unit);
      continue;
    }
    // ---- column tile it.piece of frame it.unit ----
    const int f = it.unit, tile = it.piece;
    if (threadIdx.x == 0) {
      s_ok = fused_wait(sc, f, a.err) ? 1 : 0;
      coltma_issue<N, St, WITH_S, true>(m, &tmS, &tmK, fill, f, tile, 0, a.coils, a.L);
    }
    if (f != mapped_f) {
      fused_linemap<N, C::THREADS>(s, a.lines, a.L, f, a.err);
      mapped_f = f;
    } else {
      __syncthreads();  // s_ok
    }
    const int x = tile * W + col.c;
    const bool xin = x < a.nx;
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
    bool landed = s_ok != 0;  // the same in every thread
#pragma unroll 1
    for (int c = 0; c < a.coils; ++c, ++fill) {
      landed = __syncthreads_and(coltma_wait(m.bar, fill, a.err)) && landed;
      if (threadIdx.x == 0 && c + 1 < a.coils)
        coltma_issue<N, St, WITH_S, true>(m, &tmS, &tmK, fill + 1, f, tile, c + 1, a.coils, a.L);
      const float2* kb = (fill & 1u) ? m.kb[1] : m.kb[0];
      float2 kr[C::JL][C::RL];
      float2 xr[C::J0][C::R0];
#pragma unroll
      for (int j = 0; j < C::JL; ++j)
#pragma unroll
        for (int m2 = 0; m2 < C::RL; ++m2) {
          const int row = col.krow(j, m2);
          const int l = col.okL(j) ? (int)s.map[row] : -1;
          const float2 v = l >= 0 ? kb[l * W + col.c] : make_float2(0.f, 0.f);
          kr[j][m2] = negate_if(v, a.centred && (row & 1));
        }
      const BufPair<C> bp(s.buf0, s.buf1, c);
      if constexpr (REG_TW)
        col.inv(kr, xr, bp.b, s.tw, w0);
      else
        col.inv(kr, xr, bp.b, s.tw);
      const typename St::T* sbuf = (fill & 1u) ? m.sb[1] : m.sb[0];
#pragma unroll
      for (int j = 0; j < C::J0; ++j)
#pragma unroll
        for (int n = 0; n < C::R0; ++n) {
          if (MODE == 2) {
            accr[j][n] = fmaf(xr[j][n].x, xr[j][n].x, fmaf(xr[j][n].y, xr[j][n].y, accr[j][n]));
          } else {
            const float2 sv = col.ok0(j) ? St::lds(sbuf, col.xrow(j, n) * W + col.c) : make_float2(0.f, 0.f);
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
        } else {
          g.active[f] = 0;
          g.outcome[f] = (rho == 0.0) ? CG_CONVERGED : CG_BREAKDOWN;
          g.resid[f] = (rho == 0.0) ? 0.0 : rho - rho;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// E: first pass = the column tile of k_fwd_col_tma (S_c . x, F_y, sampled
// rows into the intermediate); second pass = forward row transforms of 8 of
// a frame's coils x lines rows into y (storage type).
// ---------------------------------------------------------------------------
template <int N, class St, int TH = ColTma<N>::C::THREADS>
__global__ void __launch_bounds__(TH, ColTma<N>::MINB)
    k_forward_fused(const __grid_constant__ CUtensorMap tmS, FwdColArgs<St> a, typename St::T* y, FusedSched sc,
                    float cs) {
  using C = typename ColTma<N>::C;
  constexpr int W = C::W;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  if (smem_addr(smem_raw) & 127u) {
    if (threadIdx.x == 0) atomicOr(a.err, ERR_TIMEOUT);
    return;
  }
  const FusedSmem<N, St> fs(smem_raw, a.L, false);
  const ColTmaSmem<N, St>& m = fs.m;
  const ColSmem& s = m.s;
  __shared__ int s_ticket, s_ok;
  const C col;
  const size_t img = (size_t)N * a.nx;
  const int rows_per_frame = a.coils * a.L;
  const long total = (long)sc.frames * (sc.first_tiles + sc.second_tiles);
  for (int i = threadIdx.x; i < N; i += C::THREADS) s.tw[i] = a.tw[i];
  if (threadIdx.x == 0) {
    mbar_init(m.bar, 1);
    mbar_init(m.bar + 1, 1);
    mbar_fence_init();
  }
  __syncthreads();
  unsigned fill = 0;
  int mapped_f = -1;
  const float scale = rsqrtf((float)N);
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_ticket = (int)atomicAdd(sc.ticket, 1u);
    __syncthreads();
    const long t = s_ticket;
    if (t >= total) break;
    const StaggeredItem it = staggered_item(t, sc.frames, sc.first_tiles, sc.second_tiles, sc.lag);
    if (it.second) {  // ---- rows of frame it.unit: y = F_x(intermediate rows), kFusedRowTiles tiles of 8 ----
      if (threadIdx.x == 0) s_ok = wait_at_least(sc.done + it.unit, sc.first_tiles) ? 1 : 0;
      __syncthreads();
      if (!s_ok) {
        if (threadIdx.x == 0) atomicOr(a.err, ERR_TIMEOUT);
        continue;
      }
      for (int k = 0; k < kFusedRowTiles; ++k) {
        const int first = (it.piece * kFusedRowTiles + k) * 8;
        if (first >= rows_per_frame) break;
        const int left = rows_per_frame - first;
        if (k > 0) __syncthreads();
        fused_row_tile<N, -1, StC64, St, C>(a.tmp, y, (long)it.unit * rows_per_frame + first, left < 8 ? left : 8, s.tw,
                                            fs.tile, fs.rbuf, a.centred, cs);
      }
      continue;
    }
    // ---- column tile it.piece of frame it.unit ----
    const int f = it.unit, tile = it.piece;
    if (threadIdx.x == 0) coltma_issue<N, St, true, false>(m, &tmS, nullptr, fill, f, tile, 0, a.coils, a.L);
    if (f != mapped_f) {
      fused_linemap<N, C::THREADS>(s, a.lines, a.L, f, a.err);
      mapped_f = f;
    }
    const int x = tile * W + col.c;
    const bool xin = x < a.nx;
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
      const bool landed = __syncthreads_and(coltma_wait(m.bar, fill, a.err));
      if (threadIdx.x == 0 && c + 1 < a.coils)
        coltma_issue<N, St, true, false>(m, &tmS, nullptr, fill + 1, f, tile, c + 1, a.coils, a.L);
      const typename St::T* sbuf = (fill & 1u) ? m.sb[1] : m.sb[0];
      float2 xr[C::J0][C::R0];
      float2 kr[C::JL][C::RL];
#pragma unroll
      for (int j = 0; j < C::J0; ++j)
#pragma unroll
        for (int n = 0; n < C::R0; ++n) {
          const float2 sv = col.ok0(j) ? St::lds(sbuf, col.xrow(j, n) * W + col.c) : make_float2(0.f, 0.f);
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
    fused_count(sc.done, f);
  }
}

}  // namespace sense

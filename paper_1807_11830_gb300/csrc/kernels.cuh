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
#include "common.cuh"

namespace sense {

// shared-memory bytes of the column kernels for length N
template <int N>
constexpr size_t col_smem_bytes() {
  using C = typename Cfg<N>::C;
  return sizeof(float2) * (size_t)N            // twiddles
         + 2 * sizeof(float2) * (size_t)N * C::W  // two exchange buffers
         + 32 * sizeof(double)                 // block-sum scratch
         + sizeof(short) * (size_t)N;          // line map / sampled flags
}

template <int N>
constexpr size_t row_smem_bytes() {
  using C = typename Cfg<N>::C;
  return sizeof(float2) * (size_t)N + sizeof(float2) * (size_t)C::W * (N + 1);
}

struct ColSmem {
  float2* tw;
  float2* buf0;
  float2* buf1;
  double* red;
  short* map;
};

template <int N>
__device__ __forceinline__ ColSmem col_smem(unsigned char* base) {
  using C = typename Cfg<N>::C;
  ColSmem s;
  s.tw = reinterpret_cast<float2*>(base);
  s.buf0 = s.tw + N;
  s.buf1 = s.buf0 + N * C::W;
  s.red = reinterpret_cast<double*>(s.buf1 + N * C::W);
  s.map = reinterpret_cast<short*>(s.red + 32);
  return s;
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
  int* err;
};

template <int N, class St, int TH = Cfg<N>::C::THREADS>
__global__ void __launch_bounds__(TH) k_fwd_col(FwdColArgs<St> a) {
  using C = typename Cfg<N>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ColSmem s = col_smem<N>(smem_raw);
  const int f = blockIdx.y;
  const C col;
  const int x = blockIdx.x * C::W + col.c;
  const bool xin = x < a.nx;
  load_tw_and_linemap<N, C::THREADS>(s, a.tw, a.lines + (size_t)f * a.L, a.L, a.err);
  const size_t img = (size_t)N * a.nx;
  const float scale = rsqrtf((float)N);

  float2 xv[C::B1][C::N1];
#pragma unroll
  for (int b = 0; b < C::B1; ++b)
#pragma unroll
    for (int n1 = 0; n1 < C::N1; ++n1)
      xv[b][n1] = (col.ok1(b) && xin) ? __ldg(a.x + f * img + (size_t)col.xrow(b, n1) * a.nx + x)
                                      : make_float2(0.f, 0.f);

#pragma unroll 1
  for (int c = 0; c < a.coils; ++c) {
    float2 xr[C::B1][C::N1];
    float2 kr[C::B2][C::N2];
#pragma unroll
    for (int b = 0; b < C::B1; ++b)
#pragma unroll
      for (int n1 = 0; n1 < C::N1; ++n1) {
        float2 sv = make_float2(0.f, 0.f);
        if (col.ok1(b) && xin) sv = St::ld(a.S, c * img + (size_t)col.xrow(b, n1) * a.nx + x);
        xr[b][n1] = cmul(sv, xv[b][n1]);
      }
    col.fwd(xr, kr, (c & 1) ? s.buf1 : s.buf0, s.tw);
    float2* dst = a.tmp + ((size_t)f * a.coils + c) * a.L * a.nx;
#pragma unroll
    for (int b = 0; b < C::B2; ++b)
#pragma unroll
      for (int k2 = 0; k2 < C::N2; ++k2) {
        if (col.ok2(b) && xin) {
          const int l = s.map[col.krow(b, k2)];
          if (l >= 0) dst[(size_t)l * a.nx + x] = cscale(kr[b][k2], scale);
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
};

template <int N, int DIR, class InSt, class OutSt, int TH = Cfg<N>::C::THREADS>
__global__ void __launch_bounds__(TH)
    k_rows(RowArgs<typename InSt::T, typename OutSt::T> a) {
  using C = typename Cfg<N>::C;
  constexpr int P = N + 1;  // padded row pitch (conflict-free column access)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* tile = tw + N;
  const C col;
  const long r0 = (long)blockIdx.x * C::W;
  for (int i = threadIdx.x; i < N; i += C::THREADS) tw[i] = a.tw[i];
  for (int i = threadIdx.x; i < C::W * N; i += C::THREADS) {
    const int rr = i / N, e = i - rr * N;
    tile[rr * P + e] = (r0 + rr < a.rows) ? InSt::ld(a.in, (size_t)(r0 + rr) * N + e) : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const float scale = rsqrtf((float)N);
  float2 xr[C::B1][C::N1];
  float2 kr[C::B2][C::N2];
  float2* row = tile + col.c * P;
  if (DIR < 0) {
#pragma unroll
    for (int b = 0; b < C::B1; ++b)
#pragma unroll
      for (int n1 = 0; n1 < C::N1; ++n1) xr[b][n1] = col.ok1(b) ? row[col.xrow(b, n1)] : make_float2(0.f, 0.f);
    __syncthreads();  // the tile becomes the exchange buffer
    col.fwd(xr, kr, tile, tw);
    __syncthreads();
#pragma unroll
    for (int b = 0; b < C::B2; ++b)
#pragma unroll
      for (int k2 = 0; k2 < C::N2; ++k2)
        if (col.ok2(b)) row[col.krow(b, k2)] = cscale(kr[b][k2], scale);
  } else {
#pragma unroll
    for (int b = 0; b < C::B2; ++b)
#pragma unroll
      for (int k2 = 0; k2 < C::N2; ++k2) kr[b][k2] = col.ok2(b) ? row[col.krow(b, k2)] : make_float2(0.f, 0.f);
    __syncthreads();
    col.inv(kr, xr, tile, tw);
    __syncthreads();
#pragma unroll
    for (int b = 0; b < C::B1; ++b)
#pragma unroll
      for (int n1 = 0; n1 < C::N1; ++n1)
        if (col.ok1(b)) row[col.xrow(b, n1)] = cscale(xr[b][n1], scale);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < C::W * N; i += C::THREADS) {
    const int rr = i / N, e = i - rr * N;
    if (r0 + rr < a.rows) OutSt::st(a.out, (size_t)(r0 + rr) * N + e, tile[rr * P + e]);
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
  int* err;
  CgState cg;
};

template <int N, class St, int MODE, int TH = Cfg<N>::C::THREADS>
__global__ void __launch_bounds__(TH) k_adj_col(AdjColArgs<St> a) {
  using C = typename Cfg<N>::C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ColSmem s = col_smem<N>(smem_raw);
  const int f = blockIdx.y;
  const C col;
  const int x = blockIdx.x * C::W + col.c;
  const bool xin = x < a.nx;
  load_tw_and_linemap<N, C::THREADS>(s, a.tw, a.lines + (size_t)f * a.L, a.L, a.err);
  const size_t img = (size_t)N * a.nx;

  float2 acc[C::B1][C::N1];
  float accr[C::B1][C::N1];
#pragma unroll
  for (int b = 0; b < C::B1; ++b)
#pragma unroll
    for (int n1 = 0; n1 < C::N1; ++n1) {
      acc[b][n1] = make_float2(0.f, 0.f);
      accr[b][n1] = 0.f;
    }

#pragma unroll 1
  for (int c = 0; c < a.coils; ++c) {
    float2 xr[C::B1][C::N1];
    float2 kr[C::B2][C::N2];
    const float2* src = a.tmp + ((size_t)f * a.coils + c) * a.L * a.nx;
#pragma unroll
    for (int b = 0; b < C::B2; ++b)
#pragma unroll
      for (int k2 = 0; k2 < C::N2; ++k2) {
        float2 v = make_float2(0.f, 0.f);
        if (col.ok2(b) && xin) {
          const int l = s.map[col.krow(b, k2)];
          if (l >= 0) v = __ldg(src + (size_t)l * a.nx + x);
        }
        kr[b][k2] = v;
      }
    col.inv(kr, xr, (c & 1) ? s.buf1 : s.buf0, s.tw);
#pragma unroll
    for (int b = 0; b < C::B1; ++b)
#pragma unroll
      for (int n1 = 0; n1 < C::N1; ++n1) {
        if (MODE == 2) {
          accr[b][n1] = fmaf(xr[b][n1].x, xr[b][n1].x, fmaf(xr[b][n1].y, xr[b][n1].y, accr[b][n1]));
        } else {
          float2 sv = make_float2(0.f, 0.f);
          if (col.ok1(b) && xin) sv = St::ld(a.S, c * img + (size_t)col.xrow(b, n1) * a.nx + x);
          acc[b][n1] = cfma_conj(acc[b][n1], sv, xr[b][n1]);
        }
      }
  }

  const float scale = rsqrtf((float)N);
  float part = 0.f;
#pragma unroll
  for (int b = 0; b < C::B1; ++b)
#pragma unroll
    for (int n1 = 0; n1 < C::N1; ++n1) {
      if (!(col.ok1(b) && xin)) continue;
      const size_t idx = f * img + (size_t)col.xrow(b, n1) * a.nx + x;
      if (MODE == 2) {
        a.rss[idx] = sqrtf(accr[b][n1] * (1.0f / (float)N));
      } else {
        const float2 v = cscale(acc[b][n1], scale);
        if (MODE == 0) {
          a.x[idx] = v;
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
      if (rho > 0.0) {
        g.active[f] = 1;
        g.outcome[f] = CG_RUNNING;
        g.resid[f] = 1.0;
        atomicAdd(g.live, 1);
      } else {
        g.active[f] = 0;
        g.outcome[f] = (rho == 0.0) ? CG_CONVERGED : CG_BREAKDOWN;
        g.resid[f] = 0.0;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// E^H E, column-wise.  CG=false: out = E^H E x.
// CG=true: p = r + beta p (when p_update), q = E^H E p, Re<p,q> -> alpha.
// ---------------------------------------------------------------------------
template <class St>
struct NormalArgs {
  const float2* x;             // CG=false input
  float2* out;                 // CG=false output
  float2* p;                   // CG=true: search direction (updated in place)
  const float2* r;             // CG=true
  float2* q;                   // CG=true output
  const typename St::T* S;
  const int* lines;
  const float2* tw;
  int nx, coils, L, tiles, p_update;
  int* err;
  CgState cg;
};

template <int N, class St, bool CG, int TH = Cfg<N>::C::THREADS>
__global__ void __launch_bounds__(TH) k_normal(NormalArgs<St> a) {
  using C = typename Cfg<N>::C;
  const int f = blockIdx.y;
  if (CG && a.cg.active[f] == 0) return;  // uniform per block
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ColSmem s = col_smem<N>(smem_raw);
  const C col;
  const int x = blockIdx.x * C::W + col.c;
  const bool xin = x < a.nx;
  load_tw_and_linemap<N, C::THREADS>(s, a.tw, a.lines + (size_t)f * a.L, a.L, a.err);
  const size_t img = (size_t)N * a.nx;
  const float invN = 1.0f / (float)N;

  float beta = 0.f;
  if (CG && a.p_update) beta = (float)__ldg(a.cg.beta + f);
  float2 p[C::B1][C::N1], q[C::B1][C::N1];
#pragma unroll
  for (int b = 0; b < C::B1; ++b)
#pragma unroll
    for (int n1 = 0; n1 < C::N1; ++n1) {
      float2 v = make_float2(0.f, 0.f);
      if (col.ok1(b) && xin) {
        const size_t idx = f * img + (size_t)col.xrow(b, n1) * a.nx + x;
        if (CG) {
          v = a.p[idx];
          if (a.p_update) {
            const float2 rv = a.r[idx];
            v = make_float2(fmaf(beta, v.x, rv.x), fmaf(beta, v.y, rv.y));
            a.p[idx] = v;
          }
        } else {
          v = __ldg(a.x + idx);
        }
      }
      p[b][n1] = v;
      q[b][n1] = make_float2(0.f, 0.f);
    }

#pragma unroll 1
  for (int c = 0; c < a.coils; ++c) {
    float2 xr[C::B1][C::N1];
    float2 kr[C::B2][C::N2];
#pragma unroll
    for (int b = 0; b < C::B1; ++b)
#pragma unroll
      for (int n1 = 0; n1 < C::N1; ++n1) {
        float2 sv = make_float2(0.f, 0.f);
        if (col.ok1(b) && xin) sv = St::ld(a.S, c * img + (size_t)col.xrow(b, n1) * a.nx + x);
        xr[b][n1] = cmul(sv, p[b][n1]);
      }
    col.fwd(xr, kr, s.buf0, s.tw);
#pragma unroll
    for (int b = 0; b < C::B2; ++b)
#pragma unroll
      for (int k2 = 0; k2 < C::N2; ++k2) {
        const bool keep = col.ok2(b) && s.map[col.krow(b, k2)] >= 0;
        kr[b][k2] = keep ? cscale(kr[b][k2], invN) : make_float2(0.f, 0.f);
      }
    col.inv(kr, xr, s.buf1, s.tw);
#pragma unroll
    for (int b = 0; b < C::B1; ++b)
#pragma unroll
      for (int n1 = 0; n1 < C::N1; ++n1) {
        float2 sv = make_float2(0.f, 0.f);
        if (col.ok1(b) && xin) sv = St::ld(a.S, c * img + (size_t)col.xrow(b, n1) * a.nx + x);
        q[b][n1] = cfma_conj(q[b][n1], sv, xr[b][n1]);
      }
  }

  float part = 0.f;
#pragma unroll
  for (int b = 0; b < C::B1; ++b)
#pragma unroll
    for (int n1 = 0; n1 < C::N1; ++n1) {
      if (!(col.ok1(b) && xin)) continue;
      const size_t idx = f * img + (size_t)col.xrow(b, n1) * a.nx + x;
      if (CG) {
        a.q[idx] = q[b][n1];
        part = fmaf(p[b][n1].x, q[b][n1].x, fmaf(p[b][n1].y, q[b][n1].y, part));
      } else {
        a.out[idx] = q[b][n1];
      }
    }

  if (CG) {
    const double tot = block_sum<C::THREADS>((double)part, s.red);
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

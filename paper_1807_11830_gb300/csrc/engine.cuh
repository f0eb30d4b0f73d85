// Multi-stage mixed-radix transform of W independent length-N sequences
// ("columns" of a tile) held by one thread block, N = R_0 R_1 ... R_{S-1}.
//
// Thread layout: THREADS = T * W.  Thread (t, c) with c = tid % W the column
// and t = tid / W its phase.  With W = 16 a half-warp is one t across 16
// adjacent columns, so every shared-memory access of a half-warp is one
// 128-byte row (conflict-free) and every global access is a contiguous
// row segment.
//
// Index digits (decimation in time):
//   sample    n = n_0 P_0 + n_1 P_1 + ... + n_{S-1} P_{S-1},  P_s = prod_{j>s} R_j
//   frequency k = k_0 Q_0 + k_1 Q_1 + ... + k_{S-1} Q_{S-1},  Q_s = prod_{j<s} R_j
// Stage s runs N/R_s butterflies b = kk * P_s + r (kk < Q_s, r < P_s): an
// R_s-point DFT over n_s of the stage input, then the twiddle
// exp(-2 pi i r k_s Q_s / N) on output k_s.  Between stages the data goes
// through shared memory, laid out as row (kk + Q_s k_s) P_s + r; stage s+1
// reads row kk P_s + n_{s+1} P_{s+1} + r'.  The first stage reads registers
// (sample layout), the last writes registers (frequency layout), so an
// S-stage transform costs S-1 exchanges.  The inverse runs the stages in
// reverse with the same butterflies and rows, conjugate twiddles applied
// before each DFT.  Thread t runs butterflies b = t + T j of every stage.
#pragma once
#include "codelets.cuh"

namespace sense {

template <int... Rs>
struct Radices {
  static constexpr int S = sizeof...(Rs);
  static constexpr int r[S] = {Rs...};
  static constexpr int N = (Rs * ...);
  __host__ __device__ static constexpr int radix(int s) { return r[s]; }
  __host__ __device__ static constexpr int P(int s) {  // product of radices after s
    int p = 1;
    for (int j = s + 1; j < S; ++j) p *= r[j];
    return p;
  }
  __host__ __device__ static constexpr int Q(int s) {  // product of radices before s
    int q = 1;
    for (int j = 0; j < s; ++j) q *= r[j];
    return q;
  }
};

template <int T_, int W_, class Rad>
struct Col {
  using Radix = Rad;
  static constexpr int N = Rad::N;
  static constexpr int S = Rad::S;
  static constexpr int T = T_, W = W_;
  static constexpr int THREADS = T * W;
  static_assert(S >= 1, "at least one stage");
  static_assert(W == 4 || W == 8 || W == 16 || W == 32, "tile width");
  static_assert(THREADS % 32 == 0, "block size must be a multiple of 32");

  template <int s>
  struct St {
    static constexpr int R = Rad::radix(s);
    static constexpr int P = Rad::P(s);
    static constexpr int Q = Rad::Q(s);
    static constexpr int NB = N / R;            // butterflies of this stage
    static constexpr int J = (NB + T - 1) / T;  // butterflies per thread
    static constexpr bool FULL = (J * T == NB);
  };
  // sample-side registers (input of stage 0) and frequency-side registers
  // (output of stage S-1)
  static constexpr int J0 = St<0>::J, R0 = St<0>::R;
  static constexpr int JL = St<S - 1>::J, RL = St<S - 1>::R;
  static constexpr int P0 = St<0>::P, QL = St<S - 1>::Q;

  int t, c;
  __device__ __forceinline__ Col() : t((int)threadIdx.x / W), c((int)threadIdx.x % W) {}

  template <int s>
  __device__ __forceinline__ bool ok(int j) const {
    return St<s>::FULL || (t + T * j) < St<s>::NB;
  }
  __device__ __forceinline__ bool ok0(int j) const { return ok<0>(j); }
  __device__ __forceinline__ bool okL(int j) const { return ok<S - 1>(j); }
  // row (sample index) held in x[j][n]: n * P_0 + b
  __device__ __forceinline__ int xrow(int j, int n) const { return n * P0 + (t + T * j); }
  // frequency index held in k[j][m]: b + Q_{S-1} m
  __device__ __forceinline__ int krow(int j, int m) const { return (t + T * j) + QL * m; }
  // Shared-memory slot of (row, column).  A half-warp covers the rows of
  // G = 16 / W adjacent phases t .. t + G - 1 (t a multiple of G; G = 1 for
  // W >= 16, which is conflict-free as is).  Every stage's rows for those
  // phases either are G consecutive rows starting at a multiple of G, or
  // (the last stage, rows b*RL + n) are RL apart.  XOR-ing the low bits of
  // the row with (row / RL) mod G leaves the first kind a permutation of
  // the same G rows and spreads the second kind over all G residues, so
  // both fill 16 distinct 8-byte bank pairs.  Needs RL a multiple of G;
  // otherwise rows are stored unswizzled (correct, with some conflicts).
  __device__ __forceinline__ int sidx(int row) const {
    constexpr int G = W < 16 ? 16 / W : 1;
    if constexpr (W < 16 && RL % G == 0) {
      return (row ^ ((row / RL) & (G - 1))) * W + c;
    } else {
      return row * W + c;
    }
  }

  // ---- forward stages ----
  // stage 0: registers in, (S > 1) shared out
  __device__ __forceinline__ void fwd_first(float2 (&x)[J0][R0], float2* out, const float2* tw) const {
#pragma unroll
    for (int j = 0; j < J0; ++j) {
      if (!ok<0>(j)) continue;
      const int b = t + T * j;  // = r, kk = 0
      Dft<R0, -1>::run(x[j]);
#pragma unroll
      for (int k = 0; k < R0; ++k) {
        float2 v = x[j][k];
        if (k > 0) v = cmul(v, tw[b * k]);
        out[sidx(k * P0 + b)] = v;
      }
    }
  }

  template <int s>
  __device__ __forceinline__ void fwd_mid(const float2* in, float2* out, const float2* tw) const {
    using G = St<s>;
    constexpr int Pp = G::P * G::R;  // P_{s-1}
#pragma unroll
    for (int j = 0; j < G::J; ++j) {
      if (!ok<s>(j)) continue;
      const int b = t + T * j;
      const int kk = b / G::P, r = b - kk * G::P;
      float2 v[G::R];
#pragma unroll
      for (int n = 0; n < G::R; ++n) v[n] = in[sidx(kk * Pp + n * G::P + r)];
      Dft<G::R, -1>::run(v);
#pragma unroll
      for (int k = 0; k < G::R; ++k) {
        float2 w = v[k];
        if (k > 0) w = cmul(w, tw[r * k * G::Q]);
        out[sidx((kk + G::Q * k) * G::P + r)] = w;
      }
    }
  }

  // last stage: shared in (S > 1), registers out
  __device__ __forceinline__ void fwd_last(const float2* in, float2 (&kr)[JL][RL]) const {
    using G = St<S - 1>;
#pragma unroll
    for (int j = 0; j < JL; ++j) {
      if (!ok<S - 1>(j)) continue;
      const int kk = t + T * j;
#pragma unroll
      for (int n = 0; n < RL; ++n) kr[j][n] = in[sidx(kk * RL + n)];
      Dft<RL, -1>::run(kr[j]);
    }
  }

  template <int s>
  __device__ __forceinline__ void fwd_mids(float2* const* buf, const float2* tw) const {
    if constexpr (s < S - 1) {
      __syncthreads();
      fwd_mid<s>(buf[(s - 1) & 1], buf[s & 1], tw);
      fwd_mids<s + 1>(buf, tw);
    }
  }

  // Forward transform x (sample layout) -> k (frequency layout), unnormalised.
  // Uses buf[0], buf[1] alternately; S-1 barriers.
  __device__ __forceinline__ void fwd(float2 (&x)[J0][R0], float2 (&kr)[JL][RL], float2* const* buf,
                                      const float2* tw) const {
    if constexpr (S == 1) {
#pragma unroll
      for (int j = 0; j < J0; ++j) {
#pragma unroll
        for (int n = 0; n < R0; ++n) kr[j][n] = x[j][n];
        Dft<R0, -1>::run(kr[j]);
      }
    } else {
      fwd_first(x, buf[0], tw);
      fwd_mids<1>(buf, tw);
      __syncthreads();
      fwd_last(buf[(S - 2) & 1], kr);
    }
  }

  // ---- inverse stages (conjugate twiddles before each DFT) ----
  __device__ __forceinline__ void inv_first(float2 (&kr)[JL][RL], float2* out) const {
#pragma unroll
    for (int j = 0; j < JL; ++j) {
      if (!ok<S - 1>(j)) continue;
      const int kk = t + T * j;
      Dft<RL, 1>::run(kr[j]);
#pragma unroll
      for (int n = 0; n < RL; ++n) out[sidx(kk * RL + n)] = kr[j][n];
    }
  }

  template <int s>
  __device__ __forceinline__ void inv_mid(const float2* in, float2* out, const float2* tw) const {
    using G = St<s>;
    constexpr int Pp = G::P * G::R;
#pragma unroll
    for (int j = 0; j < G::J; ++j) {
      if (!ok<s>(j)) continue;
      const int b = t + T * j;
      const int kk = b / G::P, r = b - kk * G::P;
      float2 v[G::R];
#pragma unroll
      for (int k = 0; k < G::R; ++k) {
        float2 w = in[sidx((kk + G::Q * k) * G::P + r)];
        if (k > 0) w = cmulc(w, tw[r * k * G::Q]);
        v[k] = w;
      }
      Dft<G::R, 1>::run(v);
#pragma unroll
      for (int n = 0; n < G::R; ++n) out[sidx(kk * Pp + n * G::P + r)] = v[n];
    }
  }

  __device__ __forceinline__ void inv_last(const float2* in, float2 (&x)[J0][R0], const float2* tw) const {
#pragma unroll
    for (int j = 0; j < J0; ++j) {
      if (!ok<0>(j)) continue;
      const int b = t + T * j;
#pragma unroll
      for (int k = 0; k < R0; ++k) {
        float2 w = in[sidx(k * P0 + b)];
        if (k > 0) w = cmulc(w, tw[b * k]);
        x[j][k] = w;
      }
      Dft<R0, 1>::run(x[j]);
    }
  }

  // exchange index e = S-1 .. 2S-3 continues the alternation of the forward
  template <int s>
  __device__ __forceinline__ void inv_mids(float2* const* buf, const float2* tw) const {
    if constexpr (s >= 1) {
      __syncthreads();
      constexpr int e_in = (S - 1) + (S - 2 - s);  // exchange written by the previous inverse stage
      inv_mid<s>(buf[e_in & 1], buf[(e_in + 1) & 1], tw);
      inv_mids<s - 1>(buf, tw);
    }
  }

  // Inverse transform k (frequency layout) -> x (sample layout), unnormalised.
  // Continues the buffer alternation of fwd() so fwd followed by inv needs
  // exactly one barrier per exchange.
  __device__ __forceinline__ void inv(float2 (&kr)[JL][RL], float2 (&x)[J0][R0], float2* const* buf,
                                      const float2* tw) const {
    if constexpr (S == 1) {
#pragma unroll
      for (int j = 0; j < J0; ++j) {
#pragma unroll
        for (int n = 0; n < R0; ++n) x[j][n] = kr[j][n];
        Dft<R0, 1>::run(x[j]);
      }
    } else {
      inv_first(kr, buf[(S - 1) & 1]);
      inv_mids<S - 2>(buf, tw);
      __syncthreads();
      inv_last(buf[(2 * S - 3) & 1], x, tw);
    }
  }

  // Stage-0 (and, with three stages and T a multiple of P_1, stage-1)
  // twiddles of this thread held in registers: they depend only on the
  // thread's phase, so a kernel that runs many transforms loads them once.
  static constexpr bool TW1 = (S == 3) && (T % St<1>::P == 0);
  static constexpr int R1 = S > 1 ? St<1>::R : 2;
  struct Tw0 {
    float2 w[J0][R0 - 1];
    float2 w1[TW1 ? R1 - 1 : 1];
  };
  __device__ __forceinline__ Tw0 load_tw0(const float2* tw) const {
    Tw0 r;
#pragma unroll
    for (int j = 0; j < J0; ++j)
#pragma unroll
      for (int k = 1; k < R0; ++k) r.w[j][k - 1] = ok<0>(j) ? tw[(t + T * j) * k] : make_float2(1.f, 0.f);
    if constexpr (TW1) {
#pragma unroll
      for (int k = 1; k < R1; ++k) r.w1[k - 1] = tw[(t % St<1>::P) * k * St<1>::Q];
    }
    return r;
  }
  __device__ __forceinline__ void inv(float2 (&kr)[JL][RL], float2 (&x)[J0][R0], float2* const* buf,
                                      const float2* tw, const Tw0& w0) const {
    if constexpr (S == 1) {
      inv(kr, x, buf, tw);
    } else {
      inv_first(kr, buf[(S - 1) & 1]);
      if constexpr (TW1) {
        __syncthreads();
        using G = St<1>;
        constexpr int Pp = G::P * G::R;
        const float2* in = buf[(S - 1) & 1];
        float2* out = buf[S & 1];
#pragma unroll
        for (int j = 0; j < G::J; ++j) {
          if (!ok<1>(j)) continue;
          const int b = t + T * j;
          const int kk = b / G::P, r = b - kk * G::P;
          float2 v[G::R];
#pragma unroll
          for (int k = 0; k < G::R; ++k) {
            float2 w = in[sidx((kk + G::Q * k) * G::P + r)];
            if (k > 0) w = cmulc(w, w0.w1[k - 1]);
            v[k] = w;
          }
          Dft<G::R, 1>::run(v);
#pragma unroll
          for (int n = 0; n < G::R; ++n) out[sidx(kk * Pp + n * G::P + r)] = v[n];
        }
      } else {
        inv_mids<S - 2>(buf, tw);
      }
      __syncthreads();
      const float2* in = buf[(2 * S - 3) & 1];
#pragma unroll
      for (int j = 0; j < J0; ++j) {
        if (!ok<0>(j)) continue;
        const int b = t + T * j;
#pragma unroll
        for (int k = 0; k < R0; ++k) {
          float2 w = in[sidx(k * P0 + b)];
          if (k > 0) w = cmulc(w, w0.w[j][k - 1]);
          x[j][k] = w;
        }
        Dft<R0, 1>::run(x[j]);
      }
    }
  }
};

// ---------------------------------------------------------------------------
// Lane-major variant: the T = 16 or 32 threads of a column are consecutive
// lanes of one warp (t = tid % T, c = tid / T), so every exchange stays
// inside a warp and needs only __syncwarp().  Each column owns a region of
// CP elements per exchange buffer.  Exchange e (between stage e and stage
// e+1, in either direction) stores row `row` at Pad_e::map(row) =
// row + A_e (row >> B_e), padding chosen so that both the writing and the
// reading stage put a half-warp's 16 lanes on 16 distinct 8-byte bank pairs.
// Inter-stage twiddles come from per-stage tables tw_s[k-1][r] =
// exp(-2 pi i r k Q_s / N) (r < P_s), so lanes read consecutive entries.
// ---------------------------------------------------------------------------
template <int A_, int B_>
struct Pad {
  static constexpr int A = A_, B = B_;
  __host__ __device__ static constexpr int map(int row) { return row + A * (row >> B); }
};

template <class... Ps>
struct Pads {
  static constexpr int count = sizeof...(Ps);
};

template <int e, class L>
struct PadAt;
template <class P0, class... Ps>
struct PadAt<0, Pads<P0, Ps...>> {
  using type = P0;
};
template <int e, class P0, class... Ps>
struct PadAt<e, Pads<P0, Ps...>> {
  using type = typename PadAt<e - 1, Pads<Ps...>>::type;
};

template <int T_, int W_, class Rad, class Lay>
struct WCol {
  static constexpr int N = Rad::N;
  static constexpr int S = Rad::S;
  static constexpr int T = T_, W = W_;
  static constexpr int THREADS = T * W;
  static_assert(T == 16 || T == 32, "a column's threads must be lanes of one warp");
  static_assert(S >= 2 && Lay::count == S - 1, "one layout per exchange");
  static_assert(THREADS % 32 == 0, "block size must be a multiple of 32");

  template <int s>
  struct St {
    static constexpr int R = Rad::radix(s);
    static constexpr int P = Rad::P(s);
    static constexpr int Q = Rad::Q(s);
    static constexpr int NB = N / R;
    static constexpr int J = (NB + T - 1) / T;
    static constexpr bool FULL = (J * T == NB);
  };
  static constexpr int J0 = St<0>::J, R0 = St<0>::R;
  static constexpr int JL = St<S - 1>::J, RL = St<S - 1>::R;
  static constexpr int P0 = St<0>::P, QL = St<S - 1>::Q;

  // twiddle tables: stage s (s < S - 1) at offset twoff(s), (R_s - 1) x P_s
  __host__ __device__ static constexpr int twoff(int s) {
    int o = 0;
    for (int j = 0; j < s; ++j) o += (Rad::radix(j) - 1) * Rad::P(j);
    return o;
  }
  static constexpr int TWN = twoff(S - 1);

  // column pitch: every exchange layout fits, and CP = 2 (mod 16) so that a
  // block-wide transposing copy (two rows x eight columns per half-warp)
  // is conflict-free as well
  static constexpr int layout_rows() {
    int m = N;
    m = m > lay_size<0>() ? m : lay_size<0>();
    if constexpr (S > 2) m = m > lay_size<1>() ? m : lay_size<1>();
    if constexpr (S > 3) m = m > lay_size<2>() ? m : lay_size<2>();
    return m;
  }
  template <int e>
  static constexpr int lay_size() {
    return PadAt<e, Lay>::type::map(N - 1) + 1;
  }
  static_assert(S <= 4, "layout_rows covers up to three exchanges");
  static constexpr int CP = ((layout_rows() + 13) / 16) * 16 + 2;

  int t, c;
  __device__ __forceinline__ WCol() : t((int)threadIdx.x % T), c((int)threadIdx.x / T) {}

  template <int s>
  __device__ __forceinline__ bool ok(int j) const {
    return St<s>::FULL || (t + T * j) < St<s>::NB;
  }
  __device__ __forceinline__ bool ok0(int j) const { return ok<0>(j); }
  __device__ __forceinline__ bool okL(int j) const { return ok<S - 1>(j); }
  __device__ __forceinline__ int xrow(int j, int n) const { return n * P0 + (t + T * j); }
  __device__ __forceinline__ int krow(int j, int m) const { return (t + T * j) + QL * m; }
  template <int e>
  __device__ __forceinline__ int sidx(int row) const {
    return c * CP + PadAt<e, Lay>::type::map(row);
  }
  __device__ __forceinline__ static void sync() { __syncwarp(); }

  // ---- forward ----
  __device__ __forceinline__ void fwd_first(float2 (&x)[J0][R0], float2* out, const float2* tw) const {
#pragma unroll
    for (int j = 0; j < J0; ++j) {
      if (!ok<0>(j)) continue;
      const int b = t + T * j;  // = r (kk = 0)
      Dft<R0, -1>::run(x[j]);
#pragma unroll
      for (int k = 0; k < R0; ++k) {
        float2 v = x[j][k];
        if (k > 0) v = cmul(v, tw[twoff(0) + (k - 1) * P0 + b]);
        out[sidx<0>(k * P0 + b)] = v;
      }
    }
  }

  template <int s>
  __device__ __forceinline__ void fwd_mid(const float2* in, float2* out, const float2* tw) const {
    using G = St<s>;
    constexpr int Pp = G::P * G::R;
#pragma unroll
    for (int j = 0; j < G::J; ++j) {
      if (!ok<s>(j)) continue;
      const int b = t + T * j;
      const int kk = b / G::P, r = b - kk * G::P;
      float2 v[G::R];
#pragma unroll
      for (int n = 0; n < G::R; ++n) v[n] = in[sidx<s - 1>(kk * Pp + n * G::P + r)];
      Dft<G::R, -1>::run(v);
#pragma unroll
      for (int k = 0; k < G::R; ++k) {
        float2 w = v[k];
        if (k > 0) w = cmul(w, tw[twoff(s) + (k - 1) * G::P + r]);
        out[sidx<s>((kk + G::Q * k) * G::P + r)] = w;
      }
    }
  }

  __device__ __forceinline__ void fwd_last(const float2* in, float2 (&kr)[JL][RL]) const {
#pragma unroll
    for (int j = 0; j < JL; ++j) {
      if (!ok<S - 1>(j)) continue;
      const int kk = t + T * j;
#pragma unroll
      for (int n = 0; n < RL; ++n) kr[j][n] = in[sidx<S - 2>(kk * RL + n)];
      Dft<RL, -1>::run(kr[j]);
    }
  }

  template <int s>
  __device__ __forceinline__ void fwd_mids(float2* const* buf, const float2* tw) const {
    if constexpr (s < S - 1) {
      sync();
      fwd_mid<s>(buf[(s - 1) & 1], buf[s & 1], tw);
      fwd_mids<s + 1>(buf, tw);
    }
  }

  // x (sample layout) -> kr (frequency layout), unnormalised; buffers
  // alternate buf[0], buf[1]; tw = the stage twiddle tables
  __device__ __forceinline__ void fwd(float2 (&x)[J0][R0], float2 (&kr)[JL][RL], float2* const* buf,
                                      const float2* tw) const {
    fwd_first(x, buf[0], tw);
    fwd_mids<1>(buf, tw);
    sync();
    fwd_last(buf[(S - 2) & 1], kr);
  }

  // ---- inverse (conjugate twiddles before each DFT) ----
  __device__ __forceinline__ void inv_first(float2 (&kr)[JL][RL], float2* out) const {
#pragma unroll
    for (int j = 0; j < JL; ++j) {
      if (!ok<S - 1>(j)) continue;
      const int kk = t + T * j;
      Dft<RL, 1>::run(kr[j]);
#pragma unroll
      for (int n = 0; n < RL; ++n) out[sidx<S - 2>(kk * RL + n)] = kr[j][n];
    }
  }

  template <int s>
  __device__ __forceinline__ void inv_mid(const float2* in, float2* out, const float2* tw) const {
    using G = St<s>;
    constexpr int Pp = G::P * G::R;
#pragma unroll
    for (int j = 0; j < G::J; ++j) {
      if (!ok<s>(j)) continue;
      const int b = t + T * j;
      const int kk = b / G::P, r = b - kk * G::P;
      float2 v[G::R];
#pragma unroll
      for (int k = 0; k < G::R; ++k) {
        float2 w = in[sidx<s>((kk + G::Q * k) * G::P + r)];
        if (k > 0) w = cmulc(w, tw[twoff(s) + (k - 1) * G::P + r]);
        v[k] = w;
      }
      Dft<G::R, 1>::run(v);
#pragma unroll
      for (int n = 0; n < G::R; ++n) out[sidx<s - 1>(kk * Pp + n * G::P + r)] = v[n];
    }
  }

  __device__ __forceinline__ void inv_last(const float2* in, float2 (&x)[J0][R0], const float2* tw) const {
#pragma unroll
    for (int j = 0; j < J0; ++j) {
      if (!ok<0>(j)) continue;
      const int b = t + T * j;
#pragma unroll
      for (int k = 0; k < R0; ++k) {
        float2 w = in[sidx<0>(k * P0 + b)];
        if (k > 0) w = cmulc(w, tw[twoff(0) + (k - 1) * P0 + b]);
        x[j][k] = w;
      }
      Dft<R0, 1>::run(x[j]);
    }
  }

  template <int s>
  __device__ __forceinline__ void inv_mids(float2* const* buf, const float2* tw) const {
    if constexpr (s >= 1) {
      sync();
      constexpr int e_in = (S - 1) + (S - 2 - s);
      inv_mid<s>(buf[e_in & 1], buf[(e_in + 1) & 1], tw);
      inv_mids<s - 1>(buf, tw);
    }
  }

  // kr (frequency layout) -> x (sample layout), unnormalised; continues the
  // buffer alternation of fwd()
  __device__ __forceinline__ void inv(float2 (&kr)[JL][RL], float2 (&x)[J0][R0], float2* const* buf,
                                      const float2* tw) const {
    inv_first(kr, buf[(S - 1) & 1]);
    inv_mids<S - 2>(buf, tw);
    sync();
    inv_last(buf[(2 * S - 3) & 1], x, tw);
  }

  // Stage-0 twiddles of this lane held in registers: w[j][k-1] = table
  // entry (k - 1) P_0 + b for butterfly b = t + T j (the same for every
  // transform the lane runs), with fwd / inv overloads that use them.
  // With three stages and T a multiple of P_1, stage 1's twiddles depend on
  // the lane only (r = t mod P_1 for every butterfly of the lane): w1 holds them.
  static constexpr bool TW1 = (S == 3) && (T % St<1>::P == 0);
  static constexpr int R1 = St<1>::R;
  struct Tw0 {
    float2 w[J0][R0 - 1];
    float2 w1[TW1 ? R1 - 1 : 1];
  };
  __device__ __forceinline__ Tw0 load_tw0(const float2* tw) const {
    Tw0 r;
#pragma unroll
    for (int j = 0; j < J0; ++j)
#pragma unroll
      for (int k = 1; k < R0; ++k)
        r.w[j][k - 1] = ok<0>(j) ? tw[twoff(0) + (k - 1) * P0 + t + T * j] : make_float2(1.f, 0.f);
    if constexpr (TW1) {
#pragma unroll
      for (int k = 1; k < R1; ++k) r.w1[k - 1] = tw[twoff(1) + (k - 1) * St<1>::P + t % St<1>::P];
    }
    return r;
  }
  // stage 1 with register twiddles (forward and inverse)
  __device__ __forceinline__ void fwd_mid1(const float2* in, float2* out, const Tw0& w0) const {
    using G = St<1>;
    constexpr int Pp = G::P * G::R;
#pragma unroll
    for (int j = 0; j < G::J; ++j) {
      if (!ok<1>(j)) continue;
      const int b = t + T * j;
      const int kk = b / G::P, r = b - kk * G::P;
      float2 v[G::R];
#pragma unroll
      for (int n = 0; n < G::R; ++n) v[n] = in[sidx<0>(kk * Pp + n * G::P + r)];
      Dft<G::R, -1>::run(v);
#pragma unroll
      for (int k = 0; k < G::R; ++k) {
        float2 w = v[k];
        if (k > 0) w = cmul(w, w0.w1[k - 1]);
        out[sidx<1>((kk + G::Q * k) * G::P + r)] = w;
      }
    }
  }
  __device__ __forceinline__ void inv_mid1(const float2* in, float2* out, const Tw0& w0) const {
    using G = St<1>;
    constexpr int Pp = G::P * G::R;
#pragma unroll
    for (int j = 0; j < G::J; ++j) {
      if (!ok<1>(j)) continue;
      const int b = t + T * j;
      const int kk = b / G::P, r = b - kk * G::P;
      float2 v[G::R];
#pragma unroll
      for (int k = 0; k < G::R; ++k) {
        float2 w = in[sidx<1>((kk + G::Q * k) * G::P + r)];
        if (k > 0) w = cmulc(w, w0.w1[k - 1]);
        v[k] = w;
      }
      Dft<G::R, 1>::run(v);
#pragma unroll
      for (int n = 0; n < G::R; ++n) out[sidx<0>(kk * Pp + n * G::P + r)] = v[n];
    }
  }
  __device__ __forceinline__ void fwd(float2 (&x)[J0][R0], float2 (&kr)[JL][RL], float2* const* buf,
                                      const float2* tw, const Tw0& w0) const {
#pragma unroll
    for (int j = 0; j < J0; ++j) {
      if (!ok<0>(j)) continue;
      const int b = t + T * j;
      Dft<R0, -1>::run(x[j]);
#pragma unroll
      for (int k = 0; k < R0; ++k) {
        float2 v = x[j][k];
        if (k > 0) v = cmul(v, w0.w[j][k - 1]);
        buf[0][sidx<0>(k * P0 + b)] = v;
      }
    }
    if constexpr (TW1) {
      sync();
      fwd_mid1(buf[0], buf[1], w0);
    } else {
      fwd_mids<1>(buf, tw);
    }
    sync();
    fwd_last(buf[(S - 2) & 1], kr);
  }
  __device__ __forceinline__ void inv(float2 (&kr)[JL][RL], float2 (&x)[J0][R0], float2* const* buf,
                                      const float2* tw, const Tw0& w0) const {
    inv_first(kr, buf[(S - 1) & 1]);
    if constexpr (TW1) {
      sync();
      inv_mid1(buf[(S - 1) & 1], buf[S & 1], w0);  // S = 3: exchange e_in = 2, written to 3
    } else {
      inv_mids<S - 2>(buf, tw);
    }
    sync();
    const float2* in = buf[(2 * S - 3) & 1];
#pragma unroll
    for (int j = 0; j < J0; ++j) {
      if (!ok<0>(j)) continue;
      const int b = t + T * j;
#pragma unroll
      for (int k = 0; k < R0; ++k) {
        float2 w = in[sidx<0>(k * P0 + b)];
        if (k > 0) w = cmulc(w, w0.w[j][k - 1]);
        x[j][k] = w;
      }
      Dft<R0, 1>::run(x[j]);
    }
  }
};

template <class C>
struct is_wcol {
  static constexpr bool value = false;
};
template <int T, int W, class Rad, class Lay>
struct is_wcol<WCol<T, W, Rad, Lay>> {
  static constexpr bool value = true;
};

}  // namespace sense

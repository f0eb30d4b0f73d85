// Register-resident small DFTs ("codelets") for the mixed-radix transforms.
//
// dft<R, DIR>(v) transforms R complex values held in registers, in place and
// in natural order, without normalisation:
//     v[k] <- sum_j v[j] exp(DIR * 2 pi i j k / R),   DIR = -1 forward, +1 inverse.
// R in {1,2,3,4,5} are written out; larger R are split R = A*B in registers
// (decimation in time, A-point transforms first, then B-point ones).
// Twiddle constants of the split are evaluated at compile time by
// turn_cos / turn_sin below, so they become immediates.
#pragma once
#include <cuda_runtime.h>

namespace sense {

// ---------------------------------------------------------------------------
// Compile-time cos / sin of 2*pi*num/den.
// Quadrant reduction on the exact rational angle, reflection to [0, pi/4],
// then the Maclaurin series of sin and cos (enough terms for double
// precision on that interval: the first dropped term is below 1e-25).
// ---------------------------------------------------------------------------
constexpr double kHalfPi = 1.57079632679489661923132169163975;

__host__ __device__ constexpr double series_sin(double a) {
  double a2 = a * a, term = a, sum = a;
  for (int k = 1; k < 14; ++k) {
    term *= -a2 / (double)((2 * k) * (2 * k + 1));
    sum += term;
  }
  return sum;
}

__host__ __device__ constexpr double series_cos(double a) {
  double a2 = a * a, term = 1.0, sum = 1.0;
  for (int k = 1; k < 14; ++k) {
    term *= -a2 / (double)((2 * k - 1) * (2 * k));
    sum += term;
  }
  return sum;
}

struct CosSin { double c, s; };

// cos and sin of (pi/2) * num / den for 0 <= num <= den.
__host__ __device__ constexpr CosSin quarter_turn(long num, long den) {
  // reflect about pi/4 so the series argument stays <= pi/4
  if (2 * num > den) {
    CosSin r = {series_sin(kHalfPi * (double)(den - num) / (double)den),
                series_cos(kHalfPi * (double)(den - num) / (double)den)};
    return r;
  }
  CosSin r = {series_cos(kHalfPi * (double)num / (double)den), series_sin(kHalfPi * (double)num / (double)den)};
  return r;
}

// cos and sin of 2*pi*num/den.
__host__ __device__ constexpr CosSin turn(long num, long den) {
  long r = num % den;
  if (r < 0) r += den;
  long q = (4 * r) / den;           // quadrant
  long rem = 4 * r - q * den;       // angle within the quadrant = (pi/2) rem/den
  CosSin b = quarter_turn(rem, den);
  if (q == 0) return b;
  if (q == 1) { CosSin o = {-b.s, b.c}; return o; }
  if (q == 2) { CosSin o = {-b.c, -b.s}; return o; }
  CosSin o = {b.s, -b.c};
  return o;
}

// ---------------------------------------------------------------------------
// complex helpers on float2
// ---------------------------------------------------------------------------
// Complex add and subtract as one paired FP32 operation (add.rn.f32x2 /
// sub.rn.f32x2 on the (re, im) register pair): the same round-to-nearest
// results as two scalar operations, in one instruction.
__device__ __forceinline__ unsigned long long f2_bits(float2 a) {
  unsigned long long u;
  memcpy(&u, &a, sizeof(u));
  return u;
}
__device__ __forceinline__ float2 bits_f2(unsigned long long u) {
  float2 a;
  memcpy(&a, &u, sizeof(a));
  return a;
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return bits_f2(r);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return bits_f2(r);
}
// Element-wise paired multiply and fused multiply-add on (re, im) pairs
// (mul.rn.f32x2 / fma.rn.f32x2): the same rounding as the two scalar
// operations.  splat(s) is the pair (s, s).
__device__ __forceinline__ float2 splat(float s) { return make_float2(s, s); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return bits_f2(r);
}
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
  return bits_f2(r);
}
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// acc + conj(b) * a
__device__ __forceinline__ float2 cfma_conj(float2 acc, float2 b, float2 a) {
  return make_float2(fmaf(b.x, a.x, fmaf(b.y, a.y, acc.x)), fmaf(b.x, a.y, fmaf(-b.y, a.x, acc.y)));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return pmul(a, splat(s)); }

// Compensated (Kahan) accumulation of a coil sum, hi + lo ~ sum_c conj(b_c) a_c.
// A plain FP32 running sum rounds every step relative to the partial sum, so
// its error grows with the number of coils and, inside CG, with the iteration
// count; lo carries the low-order bits each addition drops.  The steps use
// explicit round-to-nearest operations so that nothing is contracted or
// reassociated.
// y = (the new term) - lo is formed by the fused multiply-adds that make the
// term; the Kahan step then runs on (re, im) together as three paired adds,
// so a complex term costs four FMAs and three paired instructions.
__device__ __forceinline__ void csum_fma_conj(float2& hi, float2& lo, float2 b, float2 a) {
  const float2 y = make_float2(__fmaf_rn(b.x, a.x, __fmaf_rn(b.y, a.y, -lo.x)),
                               __fmaf_rn(b.x, a.y, __fmaf_rn(-b.y, a.x, -lo.y)));
  const float2 t = cadd(hi, y);
  lo = csub(csub(t, hi), y);
  hi = t;
}
__device__ __forceinline__ float2 csum_value(float2 hi, float2 lo) { return csub(hi, lo); }
// multiply by DIR * i
template <int DIR>
__device__ __forceinline__ float2 mul_i(float2 a) {
  return DIR > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

// v *= exp(DIR * 2 pi i * E / M), with the cheap cases spelled out.
template <int M, int E, int DIR>
__device__ __forceinline__ void twiddle_const(float2& v) {
  constexpr int r = ((E % M) + M) % M;
  if constexpr (r == 0) {
    return;
  } else if constexpr (2 * r == M) {
    v = make_float2(-v.x, -v.y);
  } else if constexpr (4 * r == M) {
    v = mul_i<DIR>(v);
  } else if constexpr (4 * r == 3 * M) {
    v = mul_i<-DIR>(v);
  } else if constexpr (8 * r == M || 8 * r == 3 * M || 8 * r == 5 * M || 8 * r == 7 * M) {
    // (+-1 +- i)/sqrt(2): two adds and two multiplies
    constexpr float h = 0.70710678118654752440f;
    constexpr CosSin cs = turn(r, M);
    constexpr float c = cs.c > 0 ? 1.0f : -1.0f;
    constexpr float s = (cs.s > 0 ? 1.0f : -1.0f) * (float)DIR;
    float re = c * v.x - s * v.y;
    float im = s * v.x + c * v.y;
    v = pmul(make_float2(re, im), splat(h));
  } else {
    constexpr CosSin cs = turn(r, M);
    constexpr float c = (float)cs.c;
    constexpr float s = (float)(cs.s * DIR);
    v = make_float2(fmaf(v.x, c, -v.y * s), fmaf(v.x, s, v.y * c));
  }
}

// ---------------------------------------------------------------------------
// codelets
// ---------------------------------------------------------------------------
template <int R, int DIR>
struct Dft;

template <int DIR>
struct Dft<1, DIR> {
  __device__ __forceinline__ static void run(float2*) {}
};

template <int DIR>
struct Dft<2, DIR> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};

template <int DIR>
struct Dft<3, DIR> {
  // X1,2 = v0 - (v1+v2)/2 +- DIR i (sqrt3/2)(v1 - v2)
  __device__ __forceinline__ static void run(float2* v) {
    constexpr float h = 0.86602540378443864676f;  // sin(2 pi / 3)
    float2 s = cadd(v[1], v[2]);
    float2 d = csub(v[1], v[2]);
    float2 m = pfma(splat(-0.5f), s, v[0]);
    float2 t = mul_i<DIR>(cscale(d, h));
    v[0] = cadd(v[0], s);
    v[1] = cadd(m, t);
    v[2] = csub(m, t);
  }
};

template <int DIR>
struct Dft<4, DIR> {
  __device__ __forceinline__ static void run(float2* v) {
    float2 a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    float2 c = cadd(v[1], v[3]), d = mul_i<DIR>(csub(v[1], v[3]));
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = cadd(b, d);
    v[3] = csub(b, d);
  }
};

template <int DIR>
struct Dft<5, DIR> {
  // With w = exp(DIR 2 pi i / 5) = c1 + DIR i s1 and w^2 = c2 + DIR i s2:
  //   X1,4 = v0 + c1 (v1+v4) + c2 (v2+v3) +- DIR i [s1 (v1-v4) + s2 (v2-v3)]
  //   X2,3 = v0 + c2 (v1+v4) + c1 (v2+v3) +- DIR i [s2 (v1-v4) - s1 (v2-v3)]
  __device__ __forceinline__ static void run(float2* v) {
    constexpr CosSin w1 = turn(1, 5), w2 = turn(2, 5);
    constexpr float c1 = (float)w1.c, s1 = (float)w1.s, c2 = (float)w2.c, s2 = (float)w2.s;
    float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    float2 t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    float2 a1 = pfma(splat(c1), t1, pfma(splat(c2), t2, v[0]));
    float2 a2 = pfma(splat(c2), t1, pfma(splat(c1), t2, v[0]));
    float2 b1 = pfma(splat(s1), t3, pmul(splat(s2), t4));
    float2 b2 = pfma(splat(s2), t3, pmul(splat(-s1), t4));
    b1 = mul_i<DIR>(b1);
    b2 = mul_i<DIR>(b2);
    v[0] = cadd(v[0], cadd(t1, t2));
    v[1] = cadd(a1, b1);
    v[4] = csub(a1, b1);
    v[2] = cadd(a2, b2);
    v[3] = csub(a2, b2);
  }
};

// R = A*B in registers.  Input sample j = B*a + b; the A-point transforms run
// over a for each b, get the twiddle exp(DIR 2 pi i b ka / R), then B-point
// transforms over b give output k = ka + A*kb.
template <int A, int B, int DIR>
struct DftSplit {
  static constexpr int R = A * B;
  template <int b, int ka>
  __device__ __forceinline__ static void tw_loop(float2 (&u)[B][A]) {
    if constexpr (b < B) {
      if constexpr (ka < A) {
        twiddle_const<R, b * ka, DIR>(u[b][ka]);
        tw_loop<b, ka + 1>(u);
      } else {
        tw_loop<b + 1, 0>(u);
      }
    }
  }
  __device__ __forceinline__ static void run(float2* v) {
    float2 u[B][A];
#pragma unroll
    for (int b = 0; b < B; ++b)
#pragma unroll
      for (int a = 0; a < A; ++a) u[b][a] = v[B * a + b];
#pragma unroll
    for (int b = 0; b < B; ++b) Dft<A, DIR>::run(u[b]);
    tw_loop<0, 0>(u);
#pragma unroll
    for (int ka = 0; ka < A; ++ka) {
      float2 t[B];
#pragma unroll
      for (int b = 0; b < B; ++b) t[b] = u[b][ka];
      Dft<B, DIR>::run(t);
#pragma unroll
      for (int kb = 0; kb < B; ++kb) v[ka + A * kb] = t[kb];
    }
  }
};

template <int DIR> struct Dft<6, DIR> : DftSplit<2, 3, DIR> {};
template <int DIR> struct Dft<8, DIR> : DftSplit<4, 2, DIR> {};
template <int DIR> struct Dft<10, DIR> : DftSplit<2, 5, DIR> {};
template <int DIR> struct Dft<12, DIR> : DftSplit<4, 3, DIR> {};
template <int DIR> struct Dft<15, DIR> : DftSplit<3, 5, DIR> {};
template <int DIR> struct Dft<16, DIR> : DftSplit<4, 4, DIR> {};
template <int DIR> struct Dft<20, DIR> : DftSplit<4, 5, DIR> {};
template <int DIR> struct Dft<24, DIR> : DftSplit<8, 3, DIR> {};
template <int DIR> struct Dft<32, DIR> : DftSplit<8, 4, DIR> {};

}  // namespace sense

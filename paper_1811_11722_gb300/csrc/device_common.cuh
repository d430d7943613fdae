// Device building blocks of the lattice rule (sm_103a).
//
// Coordinates (Eq. 2): the fractional part {idx/n + Delta} is carried in
// unsigned fixed point, so the wrap-around of the fractional part is the
// natural overflow of the integer add and no floating-point floor is needed:
//   P   = floor(idx 2^64 / n)            from a 128-bit reciprocal of n
//   X   = P + D_k  (mod 2^64)            D_k = Delta_k 2^64
// FP64 path: X is used at 64 bits.  FP32 path: X is rounded to 32 bits and
// turned into a float in [1, 2) by placing its top 23 bits in the mantissa.
#pragma once

#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>

#include <cstdint>
#endif

#include "qmc_internal.h"

namespace qmc {

// --------------------------------------------------------------- indices --

// floor(idx 2^64 / n) within 1 (idx < n < 2^31): idx*rhi + hi64(idx*rlo).
__device__ __forceinline__ uint64_t frac64(uint32_t idx, const Recip& rc) {
  return (uint64_t)idx * rc.rhi + __umul64hi((uint64_t)idx, rc.rlo);
}

// Round the 64-bit fraction to 32 bits.
__device__ __forceinline__ uint32_t frac32(uint64_t p64) {
  return (uint32_t)((p64 + 0x80000000ull) >> 32);
}

// Lattice index (j g) mod n, exact (j, g < n < 2^31).
__device__ __forceinline__ uint32_t lattice_index(uint64_t j, uint32_t g, uint64_t n) {
  return (uint32_t)((j * (uint64_t)g) % n);
}

// Advance an index by a precomputed step (step < n): idx + step mod n.
__device__ __forceinline__ uint32_t index_step(uint32_t idx, uint32_t step, uint32_t n) {
  uint32_t t = idx + step;
  return t >= n ? t - n : t;
}

// ------------------------------------------------------------ arithmetic --

__device__ __forceinline__ float fma_(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_(double a, double b, double c) { return __fma_rn(a, b, c); }

// Reciprocal: hardware approximation refined by Newton-Raphson steps
// r <- r + r (1 - x r) (one step for float, two for double).
__device__ __forceinline__ float recip(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  float e = __fmaf_rn(-x, r, 1.0f);
  return __fmaf_rn(r, e, r);
}

__device__ __forceinline__ double recip(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  double e = __fma_rn(-x, r, 1.0);
  r = __fma_rn(r, e, r);
  e = __fma_rn(-x, r, 1.0);
  return __fma_rn(r, e, r);
}

// ------------------------------------------------ packed FP32 (f32x2) --
//
// sm_100-class SMs execute the same FP32 operation on both halves of a
// register pair in one instruction; each half rounds exactly as the scalar
// operation would.  The packed sector path evaluates two shifts per
// instruction where the work is a plain add, multiply or FMA.
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// 1 / x for both halves, given y = -x (the host negates F's coefficients, so
// -U^2 F comes out of the packed chains): r = rcp.approx(x), the negation an
// operand modifier of the scalar reciprocal; e = 1 - x r = fma(y, r, 1),
// small and exact before its one rounding; then the Newton step r + r e.
// These are the operations of recip(float), which returns the correctly
// rounded reciprocal (exhaustively checked over a binade).  A form that
// rounds y r - 2 ~ -1 + e to float instead would quantise e, itself about
// one ulp, and bias the values by ~1e-8.
__device__ __forceinline__ float2 recip_neg2(float2 y) {
  float2 r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.x) : "f"(-y.x));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.y) : "f"(-y.y));
  const float2 e = fma2(y, r, make_float2(1.0f, 1.0f));
  return fma2(r, e, r);
}

template <typename R>
__device__ __forceinline__ R ipow(R x, int a) {
  R p = R(1);
  int k = a < 0 ? -a : a;
  for (int q = 0; q < k; ++q) p *= x;
  return a < 0 ? recip(p) : p;
}

__device__ __forceinline__ bool finite_(float v) { return fabsf(v) < __int_as_float(0x7f800000); }
__device__ __forceinline__ bool finite_(double v) { return fabs(v) < __longlong_as_double(0x7ff0000000000000ll); }

// ------------------------------------------------------------ transforms --

// Float in [1, 2) from the top 23 bits of a 32-bit fraction (the +2^8
// rounding offset is folded into the shift table).
__device__ __forceinline__ float unit_f32(uint32_t X) { return __uint_as_float(0x3F800000u + (X >> 9)); }

// Distance of the 64-bit fraction X to the nearest integer, doubled:
// t = 2 min(x, 1 - x) in [0, 1], rounded to 52 bits.
__device__ __forceinline__ double twice_dist_f64(uint64_t X) {
  uint64_t S = X < ~X ? X : ~X;
  return __longlong_as_double((long long)(0x3FF0000000000000ull + ((S + 0x400ull) >> 11))) - 1.0;
}

// x in [0, 1) from a 64-bit fraction (truncated to 52 bits).
__device__ __forceinline__ double unit_f64(uint64_t X) {
  return __longlong_as_double((long long)(0x3FF0000000000000ull | (X >> 12))) - 1.0;
}

// Korobov z(s) on the lower half s <= 1/2: s^(alpha+1) sum_k kor[k] s^k.
template <int ALPHA, typename R>
__device__ __forceinline__ R korobov_lower(R s, const R* kor) {
  R p = kor[ALPHA];
#pragma unroll
  for (int k = ALPHA - 1; k >= 0; --k) p = fma_(p, s, kor[k]);
  R s2 = s * s;
  R sp;
  if constexpr (ALPHA == 1) sp = s2;
  else if constexpr (ALPHA == 2) sp = s2 * s;
  else if constexpr (ALPHA == 3) sp = s2 * s2;
  else {
    sp = s2 * s2;
#pragma unroll
    for (int q = 4; q <= ALPHA; ++q) sp *= s;
  }
  return sp * p;
}

template <int ALPHA, typename R>
__device__ __forceinline__ R upow(R u) {
  if constexpr (ALPHA == 1) return u;
  else if constexpr (ALPHA == 2) return u * u;
  else if constexpr (ALPHA == 3) return (u * u) * u;
  else {
    R p = u * u;
#pragma unroll
    for (int q = 3; q <= ALPHA; ++q) p *= u;
    return p;
  }
}

// Korobov z and weight from s = min(x, 1 - x).  ALPHA > 0: compile-time
// weight, unnormalised factor u^alpha (u = s(1-s)) with the constant
// (2a+1)!/(a!)^2 applied once per value by the caller.  ALPHA == 0: weight
// `alpha` at run time, each factor normalised (kor[7] = (2a+1)!/(a!)^2), which
// keeps float products of many high-weight factors in range.
template <int ALPHA, typename R>
__device__ __forceinline__ R korobov_apply(R s, bool upper, const R* kor, int alpha, R& w) {
  R zs, ua;
  const R u = fma_(-s, s, s);
  if constexpr (ALPHA > 0) {
    zs = korobov_lower<ALPHA>(s, kor);
    ua = upow<ALPHA>(u);
  } else {
    R p = kor[alpha];
    for (int k = alpha - 1; k >= 0; --k) p = fma_(p, s, kor[k]);
    R sp = s;
    for (int q = 0; q < alpha; ++q) sp *= s;
    zs = sp * p;
    ua = kor[7];
    for (int q = 0; q < alpha; ++q) ua *= u;
  }
  w *= ua;
  return upper ? R(1) - zs : zs;
}

// One coordinate of the FP32 path.  Returns the transformed coordinate z.
// Under the Korobov transform (weight `alpha` at run time) w is multiplied by
// the factor 4u = 4 s (1 - s) only: the caller raises the product of the d
// factors to the power alpha once per value (korobov_weight_rt), and the
// constant ((2a+1)!/(a!)^2 / 4^a)^d is applied in FP64 by the final pass.
template <int TR, int ALPHA>
__device__ __forceinline__ float coord_f32(uint32_t X, const float* kor, int alpha, float& w) {
  float xb = unit_f32(X);
  if constexpr (TR == TR_BAKER) {
    float t = __fmaf_rn(2.0f, xb, -3.0f);  // 2x - 1, exact
    return 1.0f - fabsf(t);
  } else if constexpr (TR == TR_KOROBOV) {
    static_assert(ALPHA == 0, "the FP32 float-coordinate path takes the Korobov weight at run time");
    float x = xb - 1.0f;                   // exact
    float s = fminf(x, 1.0f - x);          // exact
    float p = kor[alpha];
    for (int k = alpha - 1; k >= 0; --k) p = __fmaf_rn(p, s, kor[k]);
    float sp = s;
    for (int q = 0; q < alpha; ++q) sp *= s;
    const float zs = sp * p;
    w = __fmul_rn(w, 4.0f * __fmaf_rn(-s, s, s));  // 4u: an exact power of two times u
    return x > 0.5f ? 1.0f - zs : zs;
  } else {
    return xb - 1.0f;
  }
}

// The Korobov weight of the FP32 paths with a run-time alpha from the product
// w of the factors 4u: w^alpha as a double-float power (each product's
// rounding error kept exactly by an FMA and carried along), rounded once.
// Rounding u^alpha factor by factor in float is biased low (the low bits of
// a square of a float are far from uniform); one rounding of a nearly exact
// power is not.
__device__ __forceinline__ float korobov_weight_rt(float w, int alpha) {
  float hi = w, lo = 0.0f;
  for (int q = 1; q < alpha; ++q) {
    const float p = __fmul_rn(hi, w);
    const float e = __fmaf_rn(hi, w, -p);
    lo = __fmaf_rn(lo, w, e);
    hi = p;
  }
  return __fadd_rn(hi, lo);
}

// One coordinate of the FP64 path.
template <int TR, int ALPHA>
__device__ __forceinline__ double coord_f64(uint64_t X, const double* kor, int alpha, double& w) {
  if constexpr (TR == TR_BAKER) {
    return twice_dist_f64(X);              // 1 - |2x - 1| = 2 min(x, 1 - x)
  } else if constexpr (TR == TR_KOROBOV) {
    double s = 0.5 * twice_dist_f64(X);
    return korobov_apply<ALPHA>(s, (X >> 63) != 0, kor, alpha, w);
  } else {
    return unit_f64(X);
  }
}

// FP32 sector coordinates in 32-bit fixed point, on the integer pipe.
// Per point and dimension the base B is the fraction idx/n rounded to 32 bits
// plus a dither (below); per shift X = B + D wraps modulo 1 by itself, and
//   baker:  M = |(int32) X| = 2^32 min(x, 1 - x), z = M 2^-31,
//   none:   z = X 2^-32,
//   Korobov: s = M 2^-32 = min(x, 1 - x), the upper half when X >= 2^31.
// Each coordinate is rounded to float once, from the exact integer, so z
// carries a relative (not an absolute 2^-24) rounding error.  For baker and
// none the power of two goes into the polynomial coefficients (the host
// prescales them), so the float the kernel uses is M or X itself.
__device__ __forceinline__ uint32_t base32(uint64_t p64) { return (uint32_t)((p64 + 0x80000000ull) >> 32); }

// Rounding a coordinate that sits on the lattice to float repeats the same
// few rounding errors in a pattern tied to the lattice (at n ~ 2^24 the point
// spacing matches the float grid), which biases the sum.  A dither of
// [-64, 64) units of 2^-32, one per (point, dimension) from a Weyl sequence
// in j (an odd multiplier per dimension), spans the coarsest float spacing of
// M (2^7 units) and makes the rounding unbiased; it moves the point by at most
// 1.5e-8.  It is zero at j = 0, so the lattice point at the origin (a zero
// shift) stays exactly there.
__device__ __forceinline__ uint32_t dither32(uint64_t j, int i) {
  const uint32_t h = (uint32_t)j * (0x9E3779B9u ^ ((uint32_t)i * 0x632BE5AAu));
  return ((h >> 25) ^ 64u) - 64u;  // two's complement in [-64, 64); 0 for j = 0
}

// X read as a signed 32-bit integer is 2^32 (x - [x >= 1/2]), so
// |float((int32) X)| = 2^32 min(x, 1 - x), rounded once (rounding is symmetric,
// and X = 2^31, x = 1/2, converts exactly to -2^31).
//
// Korobov weight (weight 3 only).  w collects u = s(1 - s) of each dimension
// as is; the caller raises the product to the third power once per point and
// shift with korobov_weight_fx.  Cubing each factor in float instead
// (u * u * u) is biased low: rounding a square of a float, whose low bits are
// far from uniform, loses about 1e-10 per product on average, and over the
// d factors of the weight that summed to -3e-9 (d = 6) and -4.6e-9 (d = 8)
// of the integral against the FP64 rule.  The product of the d independent
// factors rounds without that bias, and its cube is formed from an exact
// square (two-product) with one final rounding.
template <int TR, int ALPHA>
__device__ __forceinline__ float coord_fx(uint32_t X, const float* kor, float& w) {
  if constexpr (TR == TR_NONE) {
    return __uint2float_rn(X);  // z 2^32
  } else {
    const float a = fabsf(__int2float_rn((int32_t)X));
    if constexpr (TR == TR_BAKER) {
      return a;  // z 2^31
    } else {
      static_assert(ALPHA == 3, "the fixed-point FP32 path takes Korobov weight 3");
      const float s = a * 0x1p-32f;
      w = __fmul_rn(w, __fmaf_rn(-s, s, s));  // the product of u = s (1 - s)
      // z = s^4 q(s) on the lower half, 1 - s^4 q(s) (one rounding) on the upper
      float q = kor[ALPHA];
#pragma unroll
      for (int k = ALPHA - 1; k >= 0; --k) q = __fmaf_rn(q, s, kor[k]);
      const float s2 = __fmul_rn(s, s);
      const float s4 = __fmul_rn(s2, s2);
      // one FMA for both halves: s^4 q + 0, or -s^4 q + 1 (the sign and the
      // addend from X's sign bit by integer operations)
      const float s4x = __uint_as_float(__float_as_uint(s4) ^ (X & 0x80000000u));
      const float c = __int_as_float(((int32_t)X >> 31) & 0x3F800000);
      return __fmaf_rn(s4x, q, c);
    }
  }
}

// coord_fx for two shifts at once: the same operations per lane (so the same
// values bit for bit) in packed f32x2 arithmetic; w holds the two products
// of the Korobov factors.
template <int TR, int ALPHA>
__device__ __forceinline__ float2 coord_fx2(uint32_t Xa, uint32_t Xb, const float* kor, float2& w) {
  if constexpr (TR == TR_NONE) {
    return make_float2(__uint2float_rn(Xa), __uint2float_rn(Xb));
  } else {
    const float2 a = make_float2(fabsf(__int2float_rn((int32_t)Xa)), fabsf(__int2float_rn((int32_t)Xb)));
    if constexpr (TR == TR_BAKER) {
      return a;
    } else {
      static_assert(ALPHA == 3, "the fixed-point FP32 path takes Korobov weight 3");
      const float2 s = mul2(a, make_float2(0x1p-32f, 0x1p-32f));
      w = mul2(w, fma2(make_float2(-s.x, -s.y), s, s));  // the products of u = s (1 - s)
      float2 q = make_float2(kor[ALPHA], kor[ALPHA]);
#pragma unroll
      for (int k = ALPHA - 1; k >= 0; --k) q = fma2(q, s, make_float2(kor[k], kor[k]));
      const float2 s2 = mul2(s, s);
      const float2 s4 = mul2(s2, s2);
      const float2 s4x = make_float2(__uint_as_float(__float_as_uint(s4.x) ^ (Xa & 0x80000000u)),
                                     __uint_as_float(__float_as_uint(s4.y) ^ (Xb & 0x80000000u)));
      const float2 c = make_float2(__int_as_float(((int32_t)Xa >> 31) & 0x3F800000),
                                   __int_as_float(((int32_t)Xb >> 31) & 0x3F800000));
      return fma2(s4x, q, c);  // s^4 q, or 1 - s^4 q on the upper half
    }
  }
}

// The Korobov-3 weight of the fixed-point path from the product w of the
// factors u: w^3 (the constant (2a+1)!/(a!)^2 per dimension is applied in
// FP64 by the final pass), as (hi + lo) w with hi + lo = w^2 exactly.
__device__ __forceinline__ float korobov_weight_fx(float w) {
  const float hi = __fmul_rn(w, w);
  const float lo = __fmaf_rn(w, w, -hi);
  return __fmaf_rn(hi, w, __fmul_rn(lo, w));
}

__device__ __forceinline__ float2 korobov_weight_fx2(float2 w) {
  const float2 hi = mul2(w, w);
  const float2 lo = fma2(w, w, mul2(hi, make_float2(-1.0f, -1.0f)));
  return fma2(hi, w, mul2(lo, w));
}

// ----------------------------------------------------------- polynomials --

// Dense polynomial of total degree K in D variables in nested Horner form:
//   K=1: c0 + sum_i l_i z_i
//   K=2: c0 + sum_i z_i (l_i + sum_{j>=i} q_ij z_j)
//   K=3: c0 + sum_i z_i (l_i + sum_{j>=i} z_j (q_ij + sum_{k>=j} c_ijk z_k))
// Coefficients in that nesting order (see the host packer).
template <int D, int K, typename R>
__device__ __forceinline__ R poly_dense(const R* c, const R* z) {
  R acc = c[0];
  if constexpr (K == 0) {
    return acc;
  } else if constexpr (K == 1) {
#pragma unroll
    for (int i = 0; i < D; ++i) acc = fma_(c[1 + i], z[i], acc);
  } else if constexpr (K == 2) {
    int off = 1;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      R r = c[off];
#pragma unroll
      for (int j = i; j < D; ++j) r = fma_(c[off + 1 + (j - i)], z[j], r);
      acc = fma_(z[i], r, acc);
      off += 1 + (D - i);
    }
  } else {
    int off = 1;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      R r = c[off];
      off += 1;
#pragma unroll
      for (int j = i; j < D; ++j) {
        R r2 = c[off];
#pragma unroll
        for (int k = j; k < D; ++k) r2 = fma_(c[off + 1 + (k - j)], z[k], r2);
        off += 1 + (D - j);
        r = fma_(z[j], r2, r);
      }
      acc = fma_(z[i], r, acc);
    }
  }
  return acc;
}

// poly_dense of degree 1 or 2 on coordinate pairs, with (c, c) coefficient
// pairs: the same operations in the same order, two shifts per instruction.
template <int D, int K>
__device__ __forceinline__ float2 poly_dense2(const float2* c, const float2* z) {
  static_assert(K == 1 || K == 2, "packed polynomials: degree 1 or 2");
  float2 acc = c[0];
  if constexpr (K == 1) {
#pragma unroll
    for (int i = 0; i < D; ++i) acc = fma2(c[1 + i], z[i], acc);
  } else {
    int off = 1;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      float2 r = c[off];
#pragma unroll
      for (int j = i; j < D; ++j) r = fma2(c[off + 1 + (j - i)], z[j], r);
      acc = fma2(z[i], r, acc);
      off += 1 + (D - i);
    }
  }
  return acc;
}

// ------------------------------------------------------------------ sums --

// Fast2Sum (Dekker): exact when |a| >= |b|; used to fold short float runs
// into a (hi, lo) pair.
__device__ __forceinline__ void fast2sum_add(float& hi, float& lo, float v) {
  float s = hi + v;
  float e = (hi - s) + v;
  hi = s;
  lo += e;
}

// fast2sum_add on two sums at once (packed f32x2), the same operations per
// lane: hi - s is an FFMA2 with -1, exact like the scalar subtraction's rounding.
__device__ __forceinline__ void fast2sum_add2(float2& hi, float2& lo, float2 v) {
  const float2 s = add2(hi, v);
  const float2 e = add2(fma2(s, make_float2(-1.0f, -1.0f), hi), v);
  hi = s;
  lo = add2(lo, e);
}

// TwoSum (Knuth): error-free for any ordering.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// (hi, lo) += (hi2, lo2) in float-float.
__device__ __forceinline__ void ff_add(float& hi, float& lo, float hi2, float lo2) {
  float s, e;
  two_sum(hi, hi2, s, e);
  e += lo + lo2;
  hi = s + e;
  lo = e - (hi - s);
}

__device__ __forceinline__ void warp_sum_ff(float& hi, float& lo) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    float h2 = __shfl_down_sync(0xffffffffu, hi, off);
    float l2 = __shfl_down_sync(0xffffffffu, lo, off);
    ff_add(hi, lo, h2, l2);
  }
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;
}

}  // namespace qmc

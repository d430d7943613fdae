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

// 1 / x for both halves, given y = -x: q = rcp.approx(y) ~ -1/x, one Newton
// step in the form q (y q - 2) = (1/x)(1 - e^2) for q = (1 + e)/y.  Taking
// -x as input (the host negates F's coefficients) leaves no negation on the
// packed path.
__device__ __forceinline__ float2 recip_neg2(float2 y) {
  float2 q;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(q.x) : "f"(y.x));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(q.y) : "f"(y.y));
  return mul2(q, fma2(y, q, make_float2(-2.0f, -2.0f)));
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

// One coordinate of the FP32 path.  Returns the transformed coordinate z; w
// is multiplied by the transform's weight factor.
template <int TR, int ALPHA>
__device__ __forceinline__ float coord_f32(uint32_t X, const float* kor, int alpha, float& w) {
  float xb = unit_f32(X);
  if constexpr (TR == TR_BAKER) {
    float t = __fmaf_rn(2.0f, xb, -3.0f);  // 2x - 1, exact
    return 1.0f - fabsf(t);
  } else if constexpr (TR == TR_KOROBOV) {
    float x = xb - 1.0f;                   // exact
    float s = fminf(x, 1.0f - x);          // exact
    return korobov_apply<ALPHA>(s, x > 0.5f, kor, alpha, w);
  } else {
    return xb - 1.0f;
  }
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

// Float-domain coordinates of the fast FP32 sector path.  With the point's
// doubled base b2 = 2 frac(idx/n) (the 32-bit fraction rounded to 23 bits and
// placed in a float mantissa, integer and FMA pipes only; doubling is exact)
// and the shift constant c = 2 Delta - 2,
// one add gives t = 2 (b + Delta) - 2 in [-2, 2), i.e. y = b + Delta in [0, 2)
// before the wrap.  (An add with one constant operand encodes directly; an
// FMA with an immediate 2 and a constant would first load the constant.)
// Then v = |t| - 1 = +-(2 {y} - 1), so the baker map is
// z = 1 - |2 {y} - 1| = 1 - |v| = min(|t|, 2 - |t|) with no wrap test at all, and
// s = min({y}, 1 - {y}) = (1 - |v|) / 2; {y} > 1/2 exactly when t and v have
// the same sign.
__device__ __forceinline__ float base2_f32(uint64_t p64) {
  const uint32_t X = frac32(p64) + 0x100u;         // round to 23 bits (wraps to 0 near 1: periodic)
  return __fmaf_rn(2.0f, unit_f32(X), -2.0f);      // 2 (x + 1) - 2 = 2x, exact
}

// The triangle coordinate from t = b2 + c.
template <int TR, int ALPHA>
__device__ __forceinline__ float coord_tri_t(float t, const float* kor, float& w) {
  if constexpr (TR == TR_NONE) {
    return __fmaf_rn(0.5f, t, t < 0.0f ? 1.0f : 0.0f);
  } else {
    if constexpr (TR == TR_BAKER) {
      // 1 - ||t| - 1| = min(|t|, 2 - |t|): one FP32 add and a min (ALU pipe),
      // and exact: |t| < 1 is returned as is, 2 - |t| is exact for |t| in [1, 2)
      const float a = fabsf(t);
      return fminf(a, 2.0f - a);
    } else {
      const float v = fabsf(t) - 1.0f;
      const float s = __fmaf_rn(-0.5f, fabsf(v), 0.5f);
      const bool upper = t * v > 0.0f;
      return korobov_apply<ALPHA>(s, upper, kor, 0, w);
    }
  }
}

template <int TR, int ALPHA>
__device__ __forceinline__ float coord_tri(float b2, float c, const float* kor, float& w) {
  return coord_tri_t<TR, ALPHA>(b2 + c, kor, w);
}

// The coordinate {y} the triangle form stands for, as a double (sampling output).
__device__ __forceinline__ double coord_tri_used(float b2, float c) {
  const double t = (double)(b2 + c);
  return 0.5 * t + (t < 0.0 ? 1.0 : 0.0);
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

// Contour-deformed (complex) sector integrands (Sec. 3: the Feynman
// prescription as a deformation of the integration contour into the complex
// plane, vanishing at the endpoints).
//
// After the periodizing transform y = z(x):
//   w_k  = y_k - i lambda y_k (1 - y_k) dF/dy_k (y)
//   J_kl = dw_k/dy_l = delta_kl - i lambda [delta_kl (1 - 2 y_k) dF/dy_k
//                                           + y_k (1 - y_k) d2F/dy_k dy_l]
//   f    = U(w)^aU F(w)^aF det J,   value = f * prod_i (transform weight)
// F (and U) are dense polynomials of degree <= 2 in nested Horner form, so
// dF/dy is a linear form read from F's coefficients at compile-time offsets,
// and -lambda d2F is a constant matrix the host tabulates after them.  J = I + i M with M real; its
// determinant comes from LU factorisation with partial pivoting done by
// conditional row swaps in registers (no dynamic register indexing).
//
// One thread evaluates one shift at a time (the per-point work, ~700 flops,
// dwarfs the index work it would share), keeping one complex matrix live.
#pragma once

#include "kernel_table.h"
#include "rule_kernels.cuh"

namespace qmc {

template <typename R>
struct Cx {
  R re, im;
};

template <typename R>
__device__ __forceinline__ Cx<R> cmul(Cx<R> a, Cx<R> b) {
  return {fma_(a.re, b.re, -a.im * b.im), fma_(a.re, b.im, a.im * b.re)};
}

template <typename R>
__device__ __forceinline__ Cx<R> crecip(Cx<R> a) {
  R den = fma_(a.re, a.re, a.im * a.im);
  R r = recip(den);
  return {a.re * r, -a.im * r};
}

template <typename R>
__device__ __forceinline__ Cx<R> cpow_int(Cx<R> z, int a) {
  Cx<R> p{R(1), R(0)};
  int k = a < 0 ? -a : a;
  for (int q = 0; q < k; ++q) p = cmul(p, z);
  return a < 0 ? crecip(p) : p;
}

// Offset of q_ij (i <= j) in the nested degree-2 layout.
__host__ __device__ constexpr int q_off(int D, int i, int j) {
  int off = 1;
  for (int a = 0; a < i; ++a) off += 1 + (D - a);
  return off + 1 + (j - i);
}
__host__ __device__ constexpr int l_off(int D, int i) {
  int off = 1;
  for (int a = 0; a < i; ++a) off += 1 + (D - a);
  return off;
}

// Complex evaluation of a dense degree-2 polynomial with real coefficients.
template <int D, typename R>
__device__ __forceinline__ Cx<R> poly2_complex(const R* c, const Cx<R>* z) {
  Cx<R> acc{c[0], R(0)};
#pragma unroll
  for (int i = 0; i < D; ++i) {
    Cx<R> r{c[l_off(D, i)], R(0)};
#pragma unroll
    for (int j = i; j < D; ++j) {
      const R q = c[q_off(D, i, j)];
      r.re = fma_(q, z[j].re, r.re);
      r.im = fma_(q, z[j].im, r.im);
    }
    // acc += z_i r, as four fused steps
    acc.re = fma_(z[i].re, r.re, acc.re);
    acc.re = fma_(-z[i].im, r.im, acc.re);
    acc.im = fma_(z[i].re, r.im, acc.im);
    acc.im = fma_(z[i].im, r.re, acc.im);
  }
  return acc;
}

// Complex evaluation of a degree-1 polynomial with real coefficients
// (nested layout c0, l_0 .. l_{D-1}).
template <int D, typename R>
__device__ __forceinline__ Cx<R> poly1_complex(const R* c, const Cx<R>* z) {
  Cx<R> acc{c[0], R(0)};
#pragma unroll
  for (int i = 0; i < D; ++i) {
    acc.re = fma_(c[1 + i], z[i].re, acc.re);
    acc.im = fma_(c[1 + i], z[i].im, acc.im);
  }
  return acc;
}

template <typename R>
__device__ __forceinline__ R cmag1(R re, R im) {
  return fabs(re) + fabs(im);
}

// det(J) for J = I + i M (M real, D x D) by LU; with PIVOT by partial
// pivoting, without it when the host has shown J strictly row diagonally
// dominant on the whole cube (then no pivoting is needed for stability).
template <int D, typename R, bool PIVOT = true>
__device__ __forceinline__ Cx<R> det_ipm(R (&M)[D][D]) {
  R ar[D][D], ai[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int q = 0; q < D; ++q) {
      ar[r][q] = (r == q) ? R(1) : R(0);
      ai[r][q] = M[r][q];
    }
  Cx<R> det{R(1), R(0)};
  bool neg = false;
#pragma unroll
  for (int c = 0; c < D; ++c) {
#pragma unroll
    for (int r = c + 1; r < (PIVOT ? D : 0); ++r) {
      const bool sw = cmag1(ar[r][c], ai[r][c]) > cmag1(ar[c][c], ai[c][c]);
      neg ^= sw;
#pragma unroll
      for (int q = c; q < D; ++q) {
        R tr = ar[c][q], ti = ai[c][q];
        ar[c][q] = sw ? ar[r][q] : tr;
        ai[c][q] = sw ? ai[r][q] : ti;
        ar[r][q] = sw ? tr : ar[r][q];
        ai[r][q] = sw ? ti : ai[r][q];
      }
    }
    const Cx<R> piv{ar[c][c], ai[c][c]};
    det = cmul(det, piv);
    const Cx<R> inv = crecip(piv);
#pragma unroll
    for (int r = c + 1; r < D; ++r) {
      const Cx<R> f = cmul(Cx<R>{ar[r][c], ai[r][c]}, inv);
#pragma unroll
      for (int q = c + 1; q < D; ++q) {  // a_rq -= f a_cq, as four fused steps
        ar[r][q] = fma_(-f.re, ar[c][q], ar[r][q]);
        ar[r][q] = fma_(f.im, ai[c][q], ar[r][q]);
        ai[r][q] = fma_(-f.re, ai[c][q], ai[r][q]);
        ai[r][q] = fma_(-f.im, ar[c][q], ai[r][q]);
      }
    }
  }
  if (neg) {
    det.re = -det.re;
    det.im = -det.im;
  }
  return det;
}

// Per-point base of coordinate i at point j.  The FAST FP32 variant takes
// the sector kernels' coordinates: the 32-bit fixed-point fraction plus the
// per-point dither, each coordinate rounded to float once from the exact
// integer (coord_fx), so that rounding is unbiased even where the lattice
// spacing matches the float grid; the other variants keep fix_base.
template <typename R, bool FAST>
__device__ __forceinline__ typename FixT<R>::T def_base(uint32_t idx, const Recip& rc, uint64_t j, int i) {
  if constexpr (FAST && sizeof(R) == 4) return sec_base<float>(idx, rc, j, i);
  else return fix_base<R>(idx, rc);
}

template <typename R, bool FAST>
__device__ __forceinline__ double def_coord_used(const RuleParams<R>& P, typename FixT<R>::T b, int k, int i) {
  if constexpr (FAST && sizeof(R) == 4) return (double)(uint32_t)(b + P.shiftx[k][i]) * 0x1p-32;
  else return coord_used<R>(b + shift_of(P, k, i));
}

// det(I + i M) - 1 without pivoting (J = I + i M strictly diagonally dominant
// on the cube, shown by the host).  The elimination runs on B = J - I with the
// identity implicit: the pivot of column c is 1 + b_cc, the updates
// b_rq -= f b_cq never touch it (c < q), and the determinant is carried as
// Delta = det - 1 through (1 + Delta)(1 + b) = 1 + (Delta + b + Delta b).
// Every rounding is then relative to a small quantity.  Eliminating on J
// itself rounds each diagonal entry, a value near 1, after every small
// update; in FP32 that made the configuration-4 integral 2e-8 too large (a
// step-by-step float emulation of the kernel, bit-identical to it on sampled
// points, put the whole bias in those updates).
template <int D, typename R>
__device__ __forceinline__ Cx<R> det_ipm_minus1(R (&M)[D][D]) {
  R br[D][D], bi[D][D];
#pragma unroll
  for (int r = 0; r < D; ++r)
#pragma unroll
    for (int q = 0; q < D; ++q) {
      br[r][q] = R(0);
      bi[r][q] = M[r][q];
    }
  Cx<R> del{R(0), R(0)};
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const Cx<R> b{br[c][c], bi[c][c]};
    const Cx<R> t = cmul(del, b);
    del.re = (del.re + b.re) + t.re;
    del.im = (del.im + b.im) + t.im;
    if (c + 1 < D) {
      const Cx<R> inv = crecip(Cx<R>{R(1) + b.re, b.im});
#pragma unroll
      for (int r = c + 1; r < D; ++r) {
        const Cx<R> f = cmul(Cx<R>{br[r][c], bi[r][c]}, inv);
#pragma unroll
        for (int q = c + 1; q < D; ++q) {  // b_rq -= f b_cq, as four fused steps
          br[r][q] = fma_(-f.re, br[c][q], br[r][q]);
          br[r][q] = fma_(f.im, bi[c][q], br[r][q]);
          bi[r][q] = fma_(-f.re, bi[c][q], bi[r][q]);
          bi[r][q] = fma_(-f.im, br[c][q], bi[r][q]);
        }
      }
    }
  }
  return del;
}

// Weighted complex value at one point and shift; *bad set when Im F(w) > 0.
// FAST: compile-time Korobov weight 3 and no pivoting (host-checked);
// otherwise the runtime transform and pivoted LU.  KU: degree of U (1 or 2),
// with cU in that degree's nested layout.  FP32 weights: the FAST variant
// multiplies the factors u = s (1 - s) and cubes the product once
// (korobov_weight_fx; constant 140^d in FP64 by the final pass), the others
// raise the product of the factors 4u to the run-time power once
// (korobov_weight_rt); both avoid the low bias of rounding u^alpha per factor.
template <typename R, int D, bool FAST = false, int KU = 2>
__device__ __forceinline__ Cx<R> deformed_value(const RuleParams<R>& P, const typename FixT<R>::T* base, int k,
                                                bool& bad) {
  R y[D];
  R wt = R(1);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    if constexpr (FAST && sizeof(R) == 4) y[i] = coord_fx<TR_KOROBOV, 3>(base[i] + P.shiftx[k][i], P.kor, wt);
    else if constexpr (FAST) y[i] = coord<R, TR_KOROBOV, 0>(base[i] + shift_of(P, k, i), P.kor, 3, wt);
    else y[i] = coord_general<R>(P, base[i] + shift_of(P, k, i), wt);
  }
  if constexpr (sizeof(R) == 4) {
    if constexpr (FAST) wt = korobov_weight_fx(wt);
    else if (P.tr == TR_KOROBOV) wt = korobov_weight_rt(wt, P.alpha);
  }
  const R* cF = P.cF;
  // gradient of F (linear form) and the contour
  R gr[D];
#pragma unroll
  for (int kk = 0; kk < D; ++kk) {
    R s = cF[l_off(D, kk)];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const int a = kk < j ? kk : j, b = kk < j ? j : kk;
      const R q = cF[q_off(D, a, b)];
      s = fma_(j == kk ? R(2) * q : q, y[j], s);
    }
    gr[kk] = s;
  }
  const R lam = P.lam;
  const R* nH = cF + kDefHessOff;  // -lambda times the Hessian of F (host table)
  Cx<R> z[D];
  R M[D][D];
#pragma unroll
  for (int kk = 0; kk < D; ++kk) {
    const R a = fma_(-y[kk], y[kk], y[kk]);  // y (1 - y)
    z[kk] = {y[kk], -lam * a * gr[kk]};
#pragma unroll
    for (int l = 0; l < D; ++l) M[kk][l] = a * nH[kk * D + l];
    M[kk][kk] = fma_(-lam * fma_(R(-2), y[kk], R(1)), gr[kk], M[kk][kk]);
  }
  // FAST (no pivoting): det J = 1 + Delta, applied as v = r + Delta r;
  // otherwise the pivoted LU's determinant
  Cx<R> dJ, dm1;
  if constexpr (FAST) dm1 = det_ipm_minus1<D, R>(M);
  else dJ = det_ipm<D, R, true>(M);
  Cx<R> U;
  if constexpr (KU == 1) U = poly1_complex<D, R>(P.cU, z);
  else U = poly2_complex<D, R>(P.cU, z);
  const Cx<R> F = poly2_complex<D, R>(cF, z);
  bad = F.im > R(0);
  Cx<R> v;
  const Cx<R> rv = (P.aU == -2 && P.aF == -1) ? crecip(cmul(cmul(U, U), F)) : cmul(cpow_int(U, P.aU), cpow_int(F, P.aF));
  if constexpr (FAST) {
    const Cx<R> t = cmul(dm1, rv);
    v = {rv.re + t.re, rv.im + t.im};
  } else {
    v = cmul(dJ, rv);
  }
  v.re *= wt;
  v.im *= wt;
  return v;
}

constexpr int kMcDeformed = 8;

template <typename R, int D, bool FAST = false, int KU = 2>
__global__ void __launch_bounds__(kThreads)
    deformed_kernel(const __grid_constant__ RuleParams<R> P, double* __restrict__ partial,
                    unsigned long long* __restrict__ counters, const SampleIO sio) {
  using FT = typename FixT<R>::T;
  if (sio.count > 0) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= sio.count) return;
    const uint64_t j = sio.j[s];
    const int k = sio.k[s];
    FT base[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      uint32_t idx = lattice_index(j, P.g[i], P.n);
      base[i] = def_base<R, FAST>(idx, P.rc, j, i);
      if (sio.idx) sio.idx[(size_t)s * D + i] = idx;
      if (sio.coord) sio.coord[(size_t)s * D + i] = def_coord_used<R, FAST>(P, base[i], k, i);
    }
    bool bad;
    Cx<R> v = deformed_value<R, D, FAST, KU>(P, base, k, bad);
    sio.values[2 * (size_t)s] = (double)v.re * P.value_scale;
    sio.values[2 * (size_t)s + 1] = (double)v.im * P.value_scale;
    return;
  }
  __shared__ double accs[2][kMcDeformed][kThreads];
  const uint32_t n = (uint32_t)P.n;
  const int mk = P.m_launch;
  for (int kk = 0; kk < kMcDeformed; ++kk) {
    accs[0][kk][threadIdx.x] = 0.0;
    accs[1][kk][threadIdx.x] = 0.0;
  }
  unsigned nbad = 0, ndef = 0;
  const uint64_t tile_pts = (uint64_t)kThreads * (uint64_t)P.L;
  for (uint64_t tile = blockIdx.x; tile < P.tiles; tile += gridDim.x) {
    const uint64_t j0 = tile * tile_pts + threadIdx.x;
    if (j0 >= P.n) continue;
    uint64_t left = (P.n - j0 + kThreads - 1) / kThreads;
    const int steps = left < (uint64_t)P.L ? (int)left : P.L;
#pragma unroll 1
    for (int kk = 0; kk < mk; ++kk) {
      uint32_t idx[D];
#pragma unroll
      for (int i = 0; i < D; ++i) idx[i] = lattice_index(j0, P.g[i], P.n);
      Acc<R> are, aim;
      are.init();
      aim.init();
#pragma unroll 1
      for (int s = 0; s < steps; ++s) {
        const uint64_t j = j0 + (uint64_t)s * kThreads;
        FT base[D];
#pragma unroll
        for (int i = 0; i < D; ++i) base[i] = def_base<R, FAST>(idx[i], P.rc, j, i);
        bool bad;
        Cx<R> v = deformed_value<R, D, FAST, KU>(P, base, kk, bad);
        ndef += bad ? 1u : 0u;
        if (P.check_finite) {
          const bool ok = finite_(v.re) && finite_(v.im);
          nbad += ok ? 0u : 1u;
          v.re = ok ? v.re : R(0);
          v.im = ok ? v.im : R(0);
        }
        are.add(v.re);
        aim.add(v.im);
#pragma unroll
        for (int i = 0; i < D; ++i) idx[i] = index_step(idx[i], P.gstep[i], n);
        if constexpr (sizeof(R) == 4) {
          if ((s & (FAST ? 0 : fold_mask_rt(P.tr))) == (FAST ? 0 : fold_mask_rt(P.tr))) {  // FAST: Korobov 3
            are.fold();
            aim.fold();
          }
        }
      }
      accs[0][kk][threadIdx.x] += are.thread_total();
      accs[1][kk][threadIdx.x] += aim.thread_total();
    }
  }
  __shared__ double red[kThreads / 32][kMcDeformed][2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int kk = 0; kk < mk; ++kk) {
    const double tr = warp_sum_d(accs[0][kk][threadIdx.x]);
    const double ti = warp_sum_d(accs[1][kk][threadIdx.x]);
    if (lane == 0) {
      red[warp][kk][0] = tr;
      red[warp][kk][1] = ti;
    }
  }
  unsigned long long b1 = warp_sum_u64((unsigned long long)nbad);
  unsigned long long b2 = warp_sum_u64((unsigned long long)ndef);
  if (lane == 0 && b1) atomicAdd(&counters[0], b1);
  if (lane == 0 && b2) atomicAdd(&counters[1], b2);
  __syncthreads();
  if (threadIdx.x < 2 * mk) {
    const int kk = threadIdx.x >> 1, part = threadIdx.x & 1;
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) s += red[w][kk][part];
    partial[((size_t)(P.k_base + kk) * P.nblk + blockIdx.x) * 2 + part] = s;
  }
}

// --------------------------------------------- packed FP32, two shifts --
//
// The FAST variant (Korobov 3, unpivoted LU, U of degree 1) for FP32 with
// two shifts per instruction: every real quantity of a (point, shift) is a
// float2 holding shifts 2p and 2p + 1, and the arithmetic is f32x2.  The
// coefficients come as (c, c) pairs from the launch parameters (cp):
// U's 1 + d linear slots, F's nested degree-2 slots, then the Hessian of F
// (2 q_kk on the diagonal) k-major, which fits for d <= kDef2DMax.
constexpr int kDef2DMax = 5;

struct Cx2 {
  float2 re, im;
};

__device__ __forceinline__ float2 neg2(float2 a) { return mul2(a, make_float2(-1.0f, -1.0f)); }

__device__ __forceinline__ Cx2 cmul2(const Cx2& a, const Cx2& b) {
  return {fma2(neg2(a.im), b.im, mul2(a.re, b.re)), fma2(a.re, b.im, mul2(a.im, b.re))};
}

// 1 / a: (re, -im) / |a|^2 with the correctly rounded packed reciprocal
__device__ __forceinline__ Cx2 crecip2(const Cx2& a) {
  const float2 rn = recip_neg2(fma2(a.re, a.re, mul2(a.im, a.im)));  // -1 / |a|^2
  return {mul2(a.re, neg2(rn)), mul2(a.im, rn)};
}

template <int D>
__device__ __forceinline__ Cx2 deformed_value2(const RuleParams<float>& P, const uint32_t* base, int p, bool& bad_a,
                                               bool& bad_b) {
  float2 y[D];
  float wa = 1.0f, wb = 1.0f;
#pragma unroll
  for (int i = 0; i < D; ++i)
    y[i] = make_float2(coord_fx<TR_KOROBOV, 3>(base[i] + P.shiftx[2 * p][i], P.kor, wa),
                       coord_fx<TR_KOROBOV, 3>(base[i] + P.shiftx[2 * p + 1][i], P.kor, wb));
  const float2* cu = P.cp;
  const float2* cf = P.cp + 1 + D;
  const float2* H = cf + poly_slots(D, 2);
  const float2 nlam = make_float2(-P.lam, -P.lam);
  const float2 one = make_float2(1.0f, 1.0f), zero = make_float2(0.0f, 0.0f);
  Cx2 z[D];
  float2 ar[D][D], ai[D][D];  // B = J - I = i M (real parts zero)
#pragma unroll
  for (int kk = 0; kk < D; ++kk) {
    float2 gr = cf[l_off(D, kk)];  // dF/dy_kk
#pragma unroll
    for (int j = 0; j < D; ++j) gr = fma2(H[kk * D + j], y[j], gr);
    const float2 na = mul2(nlam, fma2(neg2(y[kk]), y[kk], y[kk]));  // -lambda y (1 - y)
    z[kk] = {y[kk], mul2(na, gr)};
#pragma unroll
    for (int l = 0; l < D; ++l) {
      ar[kk][l] = zero;
      ai[kk][l] = mul2(na, H[kk * D + l]);
    }
    ai[kk][kk] = fma2(mul2(nlam, fma2(y[kk], make_float2(-2.0f, -2.0f), one)), gr, ai[kk][kk]);
  }
  // det J - 1 by LU without pivoting on B = J - I (J diagonally dominant,
  // shown by the host; see det_ipm_minus1 for why the identity stays implicit)
  Cx2 dm1{zero, zero};
#pragma unroll
  for (int c = 0; c < D; ++c) {
    const Cx2 b{ar[c][c], ai[c][c]};
    const Cx2 t = cmul2(dm1, b);
    dm1.re = add2(add2(dm1.re, b.re), t.re);
    dm1.im = add2(add2(dm1.im, b.im), t.im);
    if (c + 1 < D) {
      const Cx2 inv = crecip2(Cx2{add2(one, b.re), b.im});
#pragma unroll
      for (int r = c + 1; r < D; ++r) {
        const Cx2 f = cmul2(Cx2{ar[r][c], ai[r][c]}, inv);
        const float2 frn = neg2(f.re), fin = neg2(f.im);
#pragma unroll
        for (int q = c + 1; q < D; ++q) {  // a_rq -= f a_cq, as four fused steps
          ar[r][q] = fma2(frn, ar[c][q], ar[r][q]);
          ar[r][q] = fma2(f.im, ai[c][q], ar[r][q]);
          ai[r][q] = fma2(frn, ai[c][q], ai[r][q]);
          ai[r][q] = fma2(fin, ar[c][q], ai[r][q]);
        }
      }
    }
  }
  // U (degree 1) and F (degree 2) at w, real coefficients
  Cx2 U{cu[0], zero};
#pragma unroll
  for (int i = 0; i < D; ++i) {
    U.re = fma2(cu[1 + i], z[i].re, U.re);
    U.im = fma2(cu[1 + i], z[i].im, U.im);
  }
  Cx2 F{cf[0], zero};
#pragma unroll
  for (int i = 0; i < D; ++i) {
    Cx2 r{cf[l_off(D, i)], zero};
#pragma unroll
    for (int j = i; j < D; ++j) {
      const float2 q = cf[q_off(D, i, j)];
      r.re = fma2(q, z[j].re, r.re);
      r.im = fma2(q, z[j].im, r.im);
    }
    const float2 nzi = neg2(z[i].im);
    F.re = fma2(z[i].re, r.re, F.re);
    F.re = fma2(nzi, r.im, F.re);
    F.im = fma2(z[i].re, r.im, F.im);
    F.im = fma2(z[i].im, r.re, F.im);
  }
  bad_a = F.im.x > 0.0f;  // the contour left the allowed half-plane, Im F(w) > 0
  bad_b = F.im.y > 0.0f;
  const Cx2 rv = crecip2(cmul2(cmul2(U, U), F));
  const Cx2 t = cmul2(dm1, rv);
  Cx2 v{add2(rv.re, t.re), add2(rv.im, t.im)};
  const float2 w = korobov_weight_fx2(make_float2(wa, wb));  // (prod u)^3; 140^d in FP64 by the final pass
  v.re = mul2(v.re, w);
  v.im = mul2(v.im, w);
  return v;
}

template <int D>
__global__ void __launch_bounds__(kThreads, 2)  // two CTAs per SM: 128 registers, no spills at d = 5
    deformed2_kernel(const __grid_constant__ RuleParams<float> P, double* __restrict__ partial,
                     unsigned long long* __restrict__ counters, const SampleIO sio) {
  if (sio.count > 0) {  // sampling: the scalar path of the same variant, one (point, shift) per thread
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= sio.count) return;
    const uint64_t j = sio.j[s];
    const int k = sio.k[s];
    uint32_t base[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      uint32_t idx = lattice_index(j, P.g[i], P.n);
      base[i] = def_base<float, true>(idx, P.rc, j, i);
      if (sio.idx) sio.idx[(size_t)s * D + i] = idx;
      if (sio.coord) sio.coord[(size_t)s * D + i] = def_coord_used<float, true>(P, base[i], k, i);
    }
    bool bad;
    Cx<float> v = deformed_value<float, D, true, 1>(P, base, k, bad);
    sio.values[2 * (size_t)s] = (double)v.re * P.value_scale;
    sio.values[2 * (size_t)s + 1] = (double)v.im * P.value_scale;
    return;
  }
  __shared__ double accs[2][kMcDeformed][kThreads];
  const uint32_t n = (uint32_t)P.n;
  const int mk = P.m_launch;
  for (int kk = 0; kk < kMcDeformed; ++kk) {
    accs[0][kk][threadIdx.x] = 0.0;
    accs[1][kk][threadIdx.x] = 0.0;
  }
  unsigned nbad = 0, ndef = 0;
  const uint64_t tile_pts = (uint64_t)kThreads * (uint64_t)P.L;
  for (uint64_t tile = blockIdx.x; tile < P.tiles; tile += gridDim.x) {
    const uint64_t j0 = tile * tile_pts + threadIdx.x;
    if (j0 >= P.n) continue;
    uint64_t left = (P.n - j0 + kThreads - 1) / kThreads;
    const int steps = left < (uint64_t)P.L ? (int)left : P.L;
#pragma unroll 1
    for (int kk = 0; kk < mk; kk += 2) {
      const bool has_b = kk + 1 < mk;  // an odd last shift: the pair's second row is evaluated, not kept
      uint32_t idx[D];
#pragma unroll
      for (int i = 0; i < D; ++i) idx[i] = lattice_index(j0, P.g[i], P.n);
      Acc<float> are_a, aim_a, are_b, aim_b;
      are_a.init();
      aim_a.init();
      are_b.init();
      aim_b.init();
#pragma unroll 1
      for (int s = 0; s < steps; ++s) {
        const uint64_t j = j0 + (uint64_t)s * kThreads;
        uint32_t base[D];
#pragma unroll
        for (int i = 0; i < D; ++i) base[i] = def_base<float, true>(idx[i], P.rc, j, i);
        bool bad_a, bad_b;
        Cx2 v = deformed_value2<D>(P, base, kk >> 1, bad_a, bad_b);
        ndef += (bad_a ? 1u : 0u) + ((bad_b && has_b) ? 1u : 0u);
        const bool ok_a = finite_(v.re.x) && finite_(v.im.x);
        const bool ok_b = finite_(v.re.y) && finite_(v.im.y);
        nbad += (ok_a ? 0u : 1u) + ((ok_b || !has_b) ? 0u : 1u);
        are_a.add(ok_a ? v.re.x : 0.0f);
        aim_a.add(ok_a ? v.im.x : 0.0f);
        are_b.add(ok_b ? v.re.y : 0.0f);
        aim_b.add(ok_b ? v.im.y : 0.0f);
#pragma unroll
        for (int i = 0; i < D; ++i) idx[i] = index_step(idx[i], P.gstep[i], n);
        {  // Korobov-weighted values: every value into the (hi, lo) pairs
          are_a.fold();
          aim_a.fold();
          are_b.fold();
          aim_b.fold();
        }
      }
      accs[0][kk][threadIdx.x] += are_a.thread_total();
      accs[1][kk][threadIdx.x] += aim_a.thread_total();
      if (has_b) {
        accs[0][kk + 1][threadIdx.x] += are_b.thread_total();
        accs[1][kk + 1][threadIdx.x] += aim_b.thread_total();
      }
    }
  }
  __shared__ double red[kThreads / 32][kMcDeformed][2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int kk = 0; kk < mk; ++kk) {
    const double tr = warp_sum_d(accs[0][kk][threadIdx.x]);
    const double ti = warp_sum_d(accs[1][kk][threadIdx.x]);
    if (lane == 0) {
      red[warp][kk][0] = tr;
      red[warp][kk][1] = ti;
    }
  }
  unsigned long long b1 = warp_sum_u64((unsigned long long)nbad);
  unsigned long long b2 = warp_sum_u64((unsigned long long)ndef);
  if (lane == 0 && b1) atomicAdd(&counters[0], b1);
  if (lane == 0 && b2) atomicAdd(&counters[1], b2);
  __syncthreads();
  if (threadIdx.x < 2 * mk) {
    const int kk = threadIdx.x >> 1, part = threadIdx.x & 1;
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) s += red[w][kk][part];
    partial[((size_t)(P.k_base + kk) * P.nblk + blockIdx.x) * 2 + part] = s;
  }
}

}  // namespace qmc

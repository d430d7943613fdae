// Kernels of the shifted rank-1 lattice rule, Eq. (2), for one problem.
//
// Work layout.  The n points are cut into tiles of kThreads * L points; CTA b
// takes tiles b, b + gridDim.x, ...  Inside a tile, thread t takes points
// j = tile_start + t + s * kThreads, s = 0..L-1, so each warp walks a
// contiguous run of 32 points at every step, and a thread advances its d
// lattice indices by a precomputed step (kThreads g_i mod n) with one add and
// one conditional subtract per dimension.  All MC shifts of the launch are
// evaluated for a point before moving on (shift loop unrolled, one register
// accumulator per shift), so the index and fixed-point work of a point is
// shared by MC evaluations.
//
// Sums.  FP64: double accumulators.  FP32: a float run over G = 8 points is
// folded into a (hi, lo) float pair by Fast2Sum; at the end the pairs are
// reduced across the warp in float-float and across warps in double.  Each
// CTA writes its per-shift sum into a fixed slot; finalize_kernel adds the
// slots in a fixed order, so results are bit-reproducible for a given launch
// configuration.
#pragma once

#include "device_common.cuh"

namespace qmc {

constexpr int kFoldG = 8;

// Steps between folds of the FP32 run sums into their (hi, lo) pairs, as a
// mask: fold when (step & mask) == mask.  Korobov-weighted values span many
// binades (the weight vanishes at the faces), and a float run drops those
// below half an ulp of its running sum, always downward: -1.4e-9 of the
// integral at n ~ 4e6, d = 6.  They go into the pair one by one (mask 0, every
// step; the Fast2Sum keeps each value's rounding error).  Baker and untransformed
// values stay within a few binades and keep runs of kFoldG.
template <int TR>
__host__ __device__ constexpr int fold_mask() {
  return TR == TR_KOROBOV ? 0 : kFoldG - 1;
}
__device__ __forceinline__ int fold_mask_rt(int tr) { return tr == TR_KOROBOV ? 0 : kFoldG - 1; }

template <typename R>
struct Acc;

template <>
struct Acc<float> {
  float run, hi, lo;
  __device__ __forceinline__ void init() { run = hi = lo = 0.0f; }
  __device__ __forceinline__ void add(float v) { run += v; }
  __device__ __forceinline__ void fold() {
    fast2sum_add(hi, lo, run);
    run = 0.0f;
  }
  // warp-reduced total (valid in lane 0)
  __device__ __forceinline__ double warp_total() {
    fold();
    warp_sum_ff(hi, lo);
    return (double)hi + (double)lo;
  }
  // this thread's total
  __device__ __forceinline__ double thread_total() {
    fold();
    return (double)hi + (double)lo;
  }
};

template <>
struct Acc<double> {
  double run;
  __device__ __forceinline__ void init() { run = 0.0; }
  __device__ __forceinline__ void add(double v) { run += v; }
  __device__ __forceinline__ void fold() {}
  __device__ __forceinline__ double warp_total() { return warp_sum_d(run); }
  __device__ __forceinline__ double thread_total() { return run; }
};

// Fixed-point base of a coordinate for the precision at hand.
template <typename R>
struct FixT;
template <>
struct FixT<float> {
  using T = uint32_t;
};
template <>
struct FixT<double> {
  using T = uint64_t;
};

template <typename R>
__device__ __forceinline__ typename FixT<R>::T fix_base(uint32_t idx, const Recip& rc) {
  if constexpr (sizeof(R) == 4) return frac32(frac64(idx, rc));
  else return frac64(idx, rc);
}

template <typename R>
__device__ __forceinline__ typename FixT<R>::T shift_of(const RuleParams<R>& P, int k, int i) {
  if constexpr (sizeof(R) == 4) return P.shift32[k][i];
  else return P.shift64[k][i];
}

// Per-point base of the fast sector path: 32-bit fixed point (dithered) for
// FP32, 64-bit fixed point for FP64.
template <typename R>
struct SecBase;
template <>
struct SecBase<float> {
  using T = uint32_t;
};
template <>
struct SecBase<double> {
  using T = uint64_t;
};

// The weight of a value from the factors coord() collected under a run-time
// Korobov weight: FP32 raises their product to the power alpha once
// (korobov_weight_rt); FP64 factors are already the normalised weights.
template <typename R>
__device__ __forceinline__ R korobov_weight(R w, int alpha) {
  if constexpr (sizeof(R) == 4) return korobov_weight_rt(w, alpha);
  else return w;
}

template <typename R, int TR, int ALPHA>
__device__ __forceinline__ R coord(typename FixT<R>::T X, const R* kor, int alpha, R& w) {
  if constexpr (sizeof(R) == 4) return coord_f32<TR, ALPHA>(X, kor, alpha, w);
  else return coord_f64<TR, ALPHA>(X, kor, alpha, w);
}

// The coordinate a kernel used, as a double in [0, 1) (sampling output).
template <typename R>
__device__ __forceinline__ double coord_used(typename FixT<R>::T X) {
  if constexpr (sizeof(R) == 4) return (double)(unit_f32(X) - 1.0f);
  else return (double)(X >> 11) * 0x1p-53;
}

// --------------------------------------------------- sector, dense, fast --

// f = U^-2 F^-1 with U, F dense of degrees KU, KF, times the transform weight
// (other integer powers go to the general kernel, so this path has no
// per-evaluation branch).  FP32: float-domain triangle coordinates from the
// per-point bases b[i]; FP64: 64-bit fixed point.
// Polynomial policies: U and F from the nested-Horner coefficients in the
// kernel parameters (DensePolys), or as straight-line code generated for one
// plan (a policy struct written by the run-time specialiser, see jit.cu).
struct DensePolys {
  // the FP32 sector path's fixed-point shift k of dimension i
  __device__ static __forceinline__ uint32_t shift(const RuleParams<float>& P, int k, int i) { return P.shiftx[k][i]; }
  template <int D, int KU, int KF, typename R>
  __device__ static __forceinline__ void eval(const RuleParams<R>& P, const R* z, R& U, R& F) {
    U = poly_dense<D, KU>(P.cU, z);
    F = poly_dense<D, KF>(P.cF, z);
  }
  // packed: U and -F on coordinate pairs from the (c, c) pairs
  template <int D, int KU, int KF>
  __device__ static __forceinline__ void eval2(const RuleParams<float>& P, const float2* z, float2& U, float2& Fn) {
    U = poly_dense2<D, KU>(P.cp, z);
    Fn = poly_dense2<D, KF>(P.cp + poly_slots(D, KU), z);
  }
};

// Packed FP32 sector path applies to U of degree <= 1 and F of degree <= 2.
template <typename R, int KU, int KF>
constexpr bool kPacked = sizeof(R) == 4 && KU == 1 && KF == 2;

// Shifts 2p and 2p + 1 at one point: the fixed-point coordinates (integer add,
// one conversion each), U and -F as packed Horner chains, then -U^2 F and the
// reciprocal (recip_neg2) packed.
template <int D, int TR, int ALPHA, int KU, int KF, class POLY>
__device__ __forceinline__ float2 sector_value2(const RuleParams<float>& P, const uint32_t* base, int p) {
  float2 z[D];
  float2 w = make_float2(1.0f, 1.0f);
#pragma unroll
  for (int i = 0; i < D; ++i)
    z[i] = coord_fx2<TR, ALPHA>(base[i] + POLY::shift(P, 2 * p, i), base[i] + POLY::shift(P, 2 * p + 1, i), P.kor, w);
  float2 U, Fn;
  POLY::template eval2<D, KU, KF>(P, z, U, Fn);
  float2 v = recip_neg2(mul2(mul2(U, U), Fn));
  if constexpr (TR == TR_KOROBOV) v = mul2(v, korobov_weight_fx2(w));
  return v;
}

template <typename R, int D, int TR, int ALPHA, int KU, int KF, class POLY = DensePolys>
__device__ __forceinline__ R sector_value(const RuleParams<R>& P, const typename SecBase<R>::T* base, int k) {
  R z[D];
  R w = R(1);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    if constexpr (sizeof(R) == 4) z[i] = coord_fx<TR, ALPHA>(base[i] + P.shiftx[k][i], P.kor, w);
    else z[i] = coord<R, TR, ALPHA>(base[i] + shift_of(P, k, i), P.kor, P.alpha, w);
  }
  R U, F;
  POLY::template eval<D, KU, KF, R>(P, z, U, F);
  R v = recip(U * U * F);
  if constexpr (TR == TR_KOROBOV) {
    if constexpr (sizeof(R) == 4) v *= korobov_weight_fx(w);
    else v *= w;
  }
  return v;
}

// U^-2 F^-1 times the weight at one (point, shift) of the dense degree-(1, 2)
// sector path, with U and F handed back (epsilon orders need their logs).
template <typename R, int D, int TR, int ALPHA>
__device__ __forceinline__ R eps_point(const RuleParams<R>& P, const typename SecBase<R>::T* base, int k, R& U, R& F) {
  R z[D];
  R w = R(1);
#pragma unroll
  for (int i = 0; i < D; ++i) {
    if constexpr (sizeof(R) == 4) z[i] = coord_fx<TR, ALPHA>(base[i] + P.shiftx[k][i], P.kor, w);
    else z[i] = coord<R, TR, ALPHA>(base[i] + shift_of(P, k, i), P.kor, P.alpha, w);
  }
  DensePolys::template eval<D, 1, 2, R>(P, z, U, F);
  R v = recip(U * U * F);
  if constexpr (TR == TR_KOROBOV) {
    if constexpr (sizeof(R) == 4) v *= korobov_weight_fx(w);
    else v *= w;
  }
  return v;
}

// Per-point base of coordinate i at point j (FP32: 32-bit fixed point plus the
// dither of point j, dimension i; FP64: 64-bit fixed point).
template <typename R>
__device__ __forceinline__ typename SecBase<R>::T sec_base(uint32_t idx, const Recip& rc, uint64_t j, int i) {
  if constexpr (sizeof(R) == 4) return base32(frac64(idx, rc)) + dither32(j, i);
  else return frac64(idx, rc);
}

template <typename R>
__device__ __forceinline__ double sec_coord_used(const RuleParams<R>& P, typename SecBase<R>::T b, int k, int i) {
  if constexpr (sizeof(R) == 4) return (double)(uint32_t)(b + P.shiftx[k][i]) * 0x1p-32;
  else return coord_used<R>(b + shift_of(P, k, i));
}

template <typename R, int D, int TR, int ALPHA, int KU, int KF, class POLY>
__device__ void sector_sample(const RuleParams<R>& P, const SampleIO& sio) {
  using BT = typename SecBase<R>::T;
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= sio.count) return;
  uint64_t j = sio.j[s];
  int k = sio.k[s];
  BT base[D];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    uint32_t idx = lattice_index(j, P.g[i], P.n);
    base[i] = sec_base<R>(idx, P.rc, j, i);
    if (sio.idx) sio.idx[(size_t)s * D + i] = idx;
    if (sio.coord) sio.coord[(size_t)s * D + i] = sec_coord_used<R>(P, base[i], k, i);
  }
  R v = sector_value<R, D, TR, ALPHA, KU, KF, POLY>(P, base, k);
  sio.values[2 * (size_t)s] = (double)v * (double)P.value_scale;
  sio.values[2 * (size_t)s + 1] = 0.0;
}

// Block-level epilogue: per-shift warp totals -> fixed CTA slot.
template <typename R, int MC>
__device__ __forceinline__ void block_epilogue(Acc<R>* acc, int mk, unsigned nbad, const RuleParams<R>& P,
                                               double* __restrict__ partial,
                                               unsigned long long* __restrict__ counters) {
  __shared__ double red[kThreads / 32][MC];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int kk = 0; kk < MC; ++kk) {
    double t = acc[kk].warp_total();
    if (lane == 0) red[warp][kk] = t;
  }
  unsigned long long bad = warp_sum_u64((unsigned long long)nbad);
  if (lane == 0 && bad) atomicAdd(&counters[0], bad);
  __syncthreads();
  if (threadIdx.x < mk) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) s += red[w][threadIdx.x];
    size_t slot = ((size_t)(P.k_base + threadIdx.x) * P.nblk + blockIdx.x) * 2;
    partial[slot] = s;
    partial[slot + 1] = 0.0;
  }
}

// Shift rows mk..MC-1 of a partial last chunk are padded by the host with
// copies of row 0, so the unrolled shift loop carries no predicate; only the
// epilogue drops them.  CHECK: count and leave out NaN/Inf values (off when
// the host has shown U and F positive on the cube).
// SMACC (FP32 only): the per-shift Fast2Sum pairs (hi, lo) live in dynamic
// shared memory (MC * kThreads float2) and only the short float runs stay in
// registers, which frees two thirds of the accumulator registers for higher
// occupancy.
// Packed runs -> the per-shift accumulators' runs (which then fold as usual).
template <int MC, typename R>
__device__ __forceinline__ void unpack_runs(float2* run2, Acc<R>* acc) {
  if constexpr (sizeof(R) == 4) {
#pragma unroll
    for (int p = 0; p < MC / 2; ++p) {
      acc[2 * p].run += run2[p].x;
      acc[2 * p + 1].run += run2[p].y;
      run2[p] = make_float2(0.0f, 0.0f);
    }
  }
}

template <typename R, int D, int MC, int TR, int ALPHA, int KU, int KF, bool CHECK, class POLY, bool SMACC = false>
__device__ __forceinline__ void sector_body(const RuleParams<R>& P, double* __restrict__ partial,
                                            unsigned long long* __restrict__ counters, const SampleIO& sio) {
  using FT = typename FixT<R>::T;
  if (sio.count > 0) {
    sector_sample<R, D, TR, ALPHA, KU, KF, POLY>(P, sio);
    return;
  }
  const uint32_t n = (uint32_t)P.n;
  Acc<R> acc[MC];
#pragma unroll
  for (int kk = 0; kk < MC; ++kk) acc[kk].init();
  constexpr bool kSm = SMACC && sizeof(R) == 4;
  // packed path: the float runs of shifts (2p, 2p + 1) in one register pair
  constexpr bool kPack = kPacked<R, KU, KF> && MC % 2 == 0;
  float2 run2[kPack ? MC / 2 : 1];
#pragma unroll
  for (int p = 0; p < (kPack ? MC / 2 : 1); ++p) run2[p] = make_float2(0.0f, 0.0f);
  // under Korobov every value is folded on its own (fold_mask): packed on the
  // compensated pairs directly, the same operations as the scalar fold
  constexpr bool kPackFold = kPack && !kSm && TR == TR_KOROBOV;
  float2 hi2[kPackFold ? MC / 2 : 1], lo2[kPackFold ? MC / 2 : 1];
#pragma unroll
  for (int p = 0; p < (kPackFold ? MC / 2 : 1); ++p) hi2[p] = lo2[p] = make_float2(0.0f, 0.0f);
  extern __shared__ float2 accsm[];  // [MC][kThreads] (hi, lo), used when kSm
  if constexpr (kSm) {
#pragma unroll
    for (int kk = 0; kk < MC; ++kk) accsm[kk * kThreads + threadIdx.x] = make_float2(0.0f, 0.0f);
  }
  unsigned nbad = 0;
  const uint64_t tile_pts = (uint64_t)kThreads * (uint64_t)P.L;
  for (uint64_t tile = blockIdx.x; tile < P.tiles; tile += gridDim.x) {
    const uint64_t j0 = tile * tile_pts + threadIdx.x;
    if (j0 >= P.n) continue;
    uint64_t left = (P.n - j0 + kThreads - 1) / kThreads;
    const int steps = left < (uint64_t)P.L ? (int)left : P.L;
    uint32_t idx[D];
#pragma unroll
    for (int i = 0; i < D; ++i) idx[i] = lattice_index(j0, P.g[i], P.n);
    for (int s = 0; s < steps; ++s) {
      typename SecBase<R>::T base[D];
#pragma unroll
      for (int i = 0; i < D; ++i) base[i] = sec_base<R>(idx[i], P.rc, j0 + (uint64_t)s * kThreads, i);
      if constexpr (kPack) {
#pragma unroll
        for (int p = 0; p < MC / 2; ++p) {
          float2 v = sector_value2<D, TR, ALPHA, KU, KF, POLY>(P, base, p);
          if constexpr (CHECK) {
            const bool oka = finite_(v.x), okb = finite_(v.y);
            nbad += (oka || 2 * p >= P.m_launch) ? 0u : 1u;  // padded rows are not counted
            nbad += (okb || 2 * p + 1 >= P.m_launch) ? 0u : 1u;
            v = make_float2(oka ? v.x : 0.0f, okb ? v.y : 0.0f);
          }
          if constexpr (kPackFold) fast2sum_add2(hi2[p], lo2[p], v);
          else run2[p] = add2(run2[p], v);
        }
      } else {
#pragma unroll
        for (int kk = 0; kk < MC; ++kk) {
          R v = sector_value<R, D, TR, ALPHA, KU, KF, POLY>(P, base, kk);
          if constexpr (CHECK) {
            const bool ok = finite_(v);
            nbad += (ok || kk >= P.m_launch) ? 0u : 1u;  // padded rows are not counted
            v = ok ? v : R(0);
          }
          acc[kk].add(v);
        }
      }
#pragma unroll
      for (int i = 0; i < D; ++i) idx[i] = index_step(idx[i], P.gstep[i], n);
      if constexpr (sizeof(R) == 4 && !kPackFold) {
        if ((s & fold_mask<TR>()) == fold_mask<TR>()) {
          if constexpr (kPack) unpack_runs<MC>(run2, acc);
#pragma unroll
          for (int kk = 0; kk < MC; ++kk) {
            if constexpr (kSm) {
              float2 a = accsm[kk * kThreads + threadIdx.x];
              fast2sum_add(a.x, a.y, acc[kk].run);
              accsm[kk * kThreads + threadIdx.x] = a;
              acc[kk].run = 0.0f;
            } else {
              acc[kk].fold();
            }
          }
        }
      }
    }
  }
  if constexpr (kPackFold) {
#pragma unroll
    for (int p = 0; p < MC / 2; ++p) {
      acc[2 * p].hi = hi2[p].x;
      acc[2 * p].lo = lo2[p].x;
      acc[2 * p + 1].hi = hi2[p].y;
      acc[2 * p + 1].lo = lo2[p].y;
    }
  } else if constexpr (kPack) {
    unpack_runs<MC>(run2, acc);  // the last partial run
  }
  if constexpr (kSm) {
#pragma unroll
    for (int kk = 0; kk < MC; ++kk) {
      const float2 a = accsm[kk * kThreads + threadIdx.x];
      acc[kk].hi = a.x;
      acc[kk].lo = a.y;
    }
  }
  if constexpr (!CHECK) nbad = 0;
  block_epilogue<R, MC>(acc, P.m_launch, nbad, P, partial, counters);
}

template <typename R, int D, int MC, int TR, int ALPHA, int KU, int KF, bool CHECK>
__global__ void __launch_bounds__(kThreads)
    sector_kernel(const __grid_constant__ RuleParams<R> P, double* __restrict__ partial,
                  unsigned long long* __restrict__ counters, const SampleIO sio) {
  sector_body<R, D, MC, TR, ALPHA, KU, KF, CHECK, DensePolys>(P, partial, counters, sio);
}

// ------------------------------------------------ separable integrands --

// f = 1, prod (1 + c_i z_i) exp(b_i z_i) or cos(2 pi h.z), runtime d.  The
// dimension loop is not unrolled: per point and dimension the index comes
// straight from (j g_i) mod n, shared by the MC shifts of the launch.
template <typename R, int MC, int TR, int FK>
struct SepState {
  R w[MC], prod[MC], lin[MC];
  __device__ __forceinline__ void init() {
#pragma unroll
    for (int kk = 0; kk < MC; ++kk) {
      w[kk] = R(1);
      prod[kk] = R(1);
      lin[kk] = R(0);
    }
  }
  __device__ __forceinline__ void dim(const RuleParams<R>& P, typename FixT<R>::T base, int i, int kk) {
    R z = coord<R, TR, 0>(base + shift_of(P, kk, i), P.kor, P.alpha, w[kk]);
    if constexpr (FK == FK_SEPEXP) {
      prod[kk] *= fma_(P.sep_c[i], z, R(1));
      lin[kk] = fma_(P.sep_b[i], z, lin[kk]);
    } else if constexpr (FK == FK_TRIG) {
      lin[kk] = fma_(P.sep_c[i], z, lin[kk]);
    }
  }
  __device__ __forceinline__ R value(const RuleParams<R>& P, int kk) const {
    R v;
    if constexpr (FK == FK_SEPEXP) v = prod[kk] * exp(lin[kk]);
    else if constexpr (FK == FK_TRIG) v = cospi(R(2) * lin[kk]);
    else v = R(1);
    if constexpr (TR == TR_KOROBOV) v *= korobov_weight<R>(w[kk], P.alpha);
    return v;
  }
};

template <typename R, int MC, int TR, int FK>
__global__ void __launch_bounds__(kThreads)
    separable_kernel(const __grid_constant__ RuleParams<R> P, double* __restrict__ partial,
                     unsigned long long* __restrict__ counters, const SampleIO sio) {
  using FT = typename FixT<R>::T;
  if (sio.count > 0) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= sio.count) return;
    const uint64_t j = sio.j[s];
    const int k = sio.k[s];
    R w = R(1), prod = R(1), lin = R(0);
#pragma unroll 1
    for (int i = 0; i < P.d; ++i) {
      uint32_t idx = lattice_index(j, P.g[i], P.n);
      FT X = fix_base<R>(idx, P.rc) + shift_of(P, k, i);
      if (sio.idx) sio.idx[(size_t)s * P.d + i] = idx;
      if (sio.coord) sio.coord[(size_t)s * P.d + i] = coord_used<R>(X);
      R z = coord<R, TR, 0>(X, P.kor, P.alpha, w);
      if constexpr (FK == FK_SEPEXP) {
        prod *= fma_(P.sep_c[i], z, R(1));
        lin = fma_(P.sep_b[i], z, lin);
      } else if constexpr (FK == FK_TRIG) {
        lin = fma_(P.sep_c[i], z, lin);
      }
    }
    R v;
    if constexpr (FK == FK_SEPEXP) v = prod * exp(lin);
    else if constexpr (FK == FK_TRIG) v = cospi(R(2) * lin);
    else v = R(1);
    if constexpr (TR == TR_KOROBOV) v *= korobov_weight<R>(w, P.alpha);
    sio.values[2 * (size_t)s] = (double)v * P.value_scale;
    sio.values[2 * (size_t)s + 1] = 0.0;
    return;
  }
  const int mk = P.m_launch;
  Acc<R> acc[MC];
#pragma unroll
  for (int kk = 0; kk < MC; ++kk) acc[kk].init();
  unsigned nbad = 0;
  const uint64_t tile_pts = (uint64_t)kThreads * (uint64_t)P.L;
  for (uint64_t tile = blockIdx.x; tile < P.tiles; tile += gridDim.x) {
    const uint64_t j0 = tile * tile_pts + threadIdx.x;
    if (j0 >= P.n) continue;
    uint64_t left = (P.n - j0 + kThreads - 1) / kThreads;
    const int steps = left < (uint64_t)P.L ? (int)left : P.L;
    for (int s = 0; s < steps; ++s) {
      const uint64_t j = j0 + (uint64_t)s * kThreads;
      SepState<R, MC, TR, FK> st;
      st.init();
#pragma unroll 1
      for (int i = 0; i < P.d; ++i) {
        const FT base = fix_base<R>(lattice_index(j, P.g[i], P.n), P.rc);
#pragma unroll
        for (int kk = 0; kk < MC; ++kk)
          if (kk < mk) st.dim(P, base, i, kk);
      }
#pragma unroll
      for (int kk = 0; kk < MC; ++kk) {
        if (kk < mk) {
          R v = st.value(P, kk);
          if (P.check_finite) {
            bool ok = finite_(v);
            nbad += ok ? 0u : 1u;
            v = ok ? v : R(0);
          }
          acc[kk].add(v);
        }
      }
      if constexpr (sizeof(R) == 4) {
        if ((s & fold_mask<TR>()) == fold_mask<TR>()) {
#pragma unroll
          for (int kk = 0; kk < MC; ++kk) acc[kk].fold();
        }
      }
    }
  }
  block_epilogue<R, MC>(acc, mk, nbad, P, partial, counters);
}

// --------------------------------------------------- general (sparse) --

// Runtime transform for the general kernel (Korobov weight from the params,
// normalised per factor).
template <typename R>
__device__ __forceinline__ R coord_general(const RuleParams<R>& P, typename FixT<R>::T X, R& w) {
  if (P.tr == TR_BAKER) return coord<R, TR_BAKER, 0>(X, P.kor, 0, w);
  if (P.tr == TR_KOROBOV) return coord<R, TR_KOROBOV, 0>(X, P.kor, P.alpha, w);
  return coord<R, TR_NONE, 0>(X, P.kor, 0, w);
}

// Sparse monomial sum with the point's coordinates in shared memory
// (z[i * kThreads + threadIdx.x]).
template <typename R>
__device__ __forceinline__ R sparse_eval(const SparsePoly<R>& Q, const R* z, int d) {
  R acc = R(0);
#pragma unroll 1
  for (int t = 0; t < Q.nterms; ++t) {
    R p = Q.coef[t];
#pragma unroll 1
    for (int i = 0; i < d; ++i) {
      const int e = Q.expo[t][i];
      const R zi = z[i * kThreads + threadIdx.x];
      for (int q = 0; q < e; ++q) p *= zi;
    }
    acc += p;
  }
  return acc;
}

// U^aU F^aF for any degree and d <= QMC_DMAX, everything at run time; the
// per-thread coordinates and per-shift accumulators live in shared memory.
template <typename R>
__device__ __forceinline__ R general_eval(const GeneralParams<R>& G, uint64_t j, int k, R* zsh,
                                          uint64_t* idx_out, double* coord_out, R& U, R& F) {
  const RuleParams<R>& P = G.base;
  R w = R(1);
#pragma unroll 1
  for (int i = 0; i < P.d; ++i) {
    uint32_t idx = lattice_index(j, P.g[i], P.n);
    typename FixT<R>::T X = fix_base<R>(idx, P.rc) + shift_of(P, k, i);
    if (idx_out) idx_out[i] = idx;
    if (coord_out) coord_out[i] = coord_used<R>(X);
    zsh[i * kThreads + threadIdx.x] = coord_general<R>(P, X, w);
  }
  U = sparse_eval(G.U, zsh, P.d);
  F = sparse_eval(G.F, zsh, P.d);
  if constexpr (sizeof(R) == 4) {
    if (P.tr == TR_KOROBOV) w = korobov_weight_rt(w, P.alpha);
  }
  return ipow(U, P.aU) * ipow(F, P.aF) * w;
}

template <typename R>
__device__ __forceinline__ R general_value(const GeneralParams<R>& G, uint64_t j, int k, R* zsh,
                                           uint64_t* idx_out, double* coord_out) {
  R U, F;
  return general_eval<R>(G, j, k, zsh, idx_out, coord_out, U, F);
}

template <typename R, int MC>
__global__ void __launch_bounds__(kThreads)
    general_kernel(const __grid_constant__ GeneralParams<R> G, double* __restrict__ partial,
                   unsigned long long* __restrict__ counters, const SampleIO sio) {
  __shared__ R zsh[QMC_DMAX * kThreads];
  const RuleParams<R>& P = G.base;
  if (sio.count > 0) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= sio.count) return;
    R v = general_value<R>(G, sio.j[s], sio.k[s], zsh, sio.idx ? sio.idx + (size_t)s * P.d : nullptr,
                           sio.coord ? sio.coord + (size_t)s * P.d : nullptr);
    sio.values[2 * (size_t)s] = (double)v * P.value_scale;
    sio.values[2 * (size_t)s + 1] = 0.0;
    return;
  }
  const int mk = P.m_launch;
  Acc<R> acc[MC];
#pragma unroll
  for (int kk = 0; kk < MC; ++kk) acc[kk].init();
  unsigned nbad = 0;
  const uint64_t tile_pts = (uint64_t)kThreads * (uint64_t)P.L;
  for (uint64_t tile = blockIdx.x; tile < P.tiles; tile += gridDim.x) {
    const uint64_t j0 = tile * tile_pts + threadIdx.x;
    if (j0 >= P.n) continue;
    uint64_t left = (P.n - j0 + kThreads - 1) / kThreads;
    const int steps = left < (uint64_t)P.L ? (int)left : P.L;
    for (int s = 0; s < steps; ++s) {
      const uint64_t j = j0 + (uint64_t)s * kThreads;
#pragma unroll
      for (int kk = 0; kk < MC; ++kk) {
        if (kk < mk) {
          R v = general_value<R>(G, j, kk, zsh, nullptr, nullptr);
          if (P.check_finite) {
            bool ok = finite_(v);
            nbad += ok ? 0u : 1u;
            v = ok ? v : R(0);
          }
          acc[kk].add(v);
        }
      }
      if constexpr (sizeof(R) == 4) {
        if ((s & fold_mask_rt(P.tr)) == fold_mask_rt(P.tr)) {
#pragma unroll
          for (int kk = 0; kk < MC; ++kk) acc[kk].fold();
        }
      }
    }
  }
  block_epilogue<R, MC>(acc, mk, nbad, P, partial, counters);
}


// ------------------------------------------- epsilon expansion of Eq. (7) --
//
// With regulated powers U^(aU + bU eps) F^(aF + bF eps) the integrand is
// sum_k eps^k f_k, f_k = U^aU F^aF L^k / k!, L = bU log U + bF log F.  One
// pass computes the point, the transform, U and F once and accumulates the
// NE coefficient integrands f_0..f_{NE-1} for MC shifts (NE * MC sums);
// f_k = f_{k-1} L / k.  Orders beyond P.eps_orders are evaluated but never
// written back.  Every order counts and leaves out its own NaN/Inf values (L
// is NaN where U or F is negative).

template <typename R>
__device__ __forceinline__ R log_(R x) {
  if constexpr (sizeof(R) == 4) return logf(x);
  else return log(x);
}

// Per-(order, shift) warp totals -> fixed CTA slots; per-order bad counts.
template <typename R, int MC, int NE>
__device__ __forceinline__ void eps_epilogue(Acc<R> (&acc)[NE][MC], const unsigned (&nbad)[NE],
                                             const RuleParams<R>& P, double* __restrict__ partial,
                                             unsigned long long* __restrict__ counters) {
  __shared__ double red[kThreads / 32][NE * MC];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 0; o < NE; ++o) {
#pragma unroll
    for (int kk = 0; kk < MC; ++kk) {
      double t = acc[o][kk].warp_total();
      if (lane == 0) red[warp][o * MC + kk] = t;
    }
    unsigned long long bad = warp_sum_u64((unsigned long long)nbad[o]);
    if (lane == 0 && bad && o < P.eps_orders) atomicAdd(&counters[2 * o], bad);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < NE * MC; t += kThreads) {
    const int o = t / MC, kk = t % MC;
    if (o >= P.eps_orders || kk >= P.m_launch) continue;
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) s += red[w][t];
    size_t slot = (((size_t)o * P.m_total + P.k_base + kk) * P.nblk + blockIdx.x) * 2;
    partial[slot] = s;
    partial[slot + 1] = 0.0;
  }
}

// Adds order values f_0..f_{NE-1} at one (point, shift) to the sums.
template <typename R, int MC, int NE>
__device__ __forceinline__ void eps_add(Acc<R> (&acc)[NE][MC], unsigned (&nbad)[NE], int kk, R v, R L,
                                        const RuleParams<R>& P, bool counted) {
#pragma unroll
  for (int o = 0; o < NE; ++o) {
    const bool ok = finite_(v);
    nbad[o] += (ok || !counted) ? 0u : 1u;
    acc[o][kk].add(ok ? v : R(0));
    if (o + 1 < NE) v = v * L * P.eps_inv[o];
  }
}

template <typename R, int MC, int NE>
__device__ __forceinline__ void eps_fold(Acc<R> (&acc)[NE][MC]) {
#pragma unroll
  for (int o = 0; o < NE; ++o)
#pragma unroll
    for (int kk = 0; kk < MC; ++kk) acc[o][kk].fold();
}

// Dense U (degree 1), F (degree 2), U^-2 F^-1 at eps = 0, d = D, baker or
// Korobov-3: the coordinates of the fast sector path.
template <typename R, int D, int MC, int NE, int TR, int ALPHA>
__global__ void __launch_bounds__(kThreads)
    eps_kernel(const __grid_constant__ RuleParams<R> P, double* __restrict__ partial,
               unsigned long long* __restrict__ counters, const SampleIO sio) {
  using BT = typename SecBase<R>::T;
  if (sio.count > 0) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= sio.count) return;
    const uint64_t j = sio.j[s];
    const int k = sio.k[s];
    BT base[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      uint32_t idx = lattice_index(j, P.g[i], P.n);
      base[i] = sec_base<R>(idx, P.rc, j, i);
      if (sio.idx) sio.idx[(size_t)s * D + i] = idx;
      if (sio.coord) sio.coord[(size_t)s * D + i] = sec_coord_used<R>(P, base[i], k, i);
    }
    R U, F;
    R v = eps_point<R, D, TR, ALPHA>(P, base, k, U, F);
    const R L = P.eps_b[0] * log_(U) + P.eps_b[1] * log_(F);
    for (int o = 0; o < P.eps_orders; ++o) {
      sio.values[(size_t)s * sio.stride + o] = (double)v * P.value_scale;
      v = v * L * P.eps_inv[o];
    }
    return;
  }
  const uint32_t n = (uint32_t)P.n;
  Acc<R> acc[NE][MC];
#pragma unroll
  for (int o = 0; o < NE; ++o)
#pragma unroll
    for (int kk = 0; kk < MC; ++kk) acc[o][kk].init();
  unsigned nbad[NE];
#pragma unroll
  for (int o = 0; o < NE; ++o) nbad[o] = 0;
  const uint64_t tile_pts = (uint64_t)kThreads * (uint64_t)P.L;
  for (uint64_t tile = blockIdx.x; tile < P.tiles; tile += gridDim.x) {
    const uint64_t j0 = tile * tile_pts + threadIdx.x;
    if (j0 >= P.n) continue;
    uint64_t left = (P.n - j0 + kThreads - 1) / kThreads;
    const int steps = left < (uint64_t)P.L ? (int)left : P.L;
    uint32_t idx[D];
#pragma unroll
    for (int i = 0; i < D; ++i) idx[i] = lattice_index(j0, P.g[i], P.n);
    for (int s = 0; s < steps; ++s) {
      BT base[D];
#pragma unroll
      for (int i = 0; i < D; ++i) base[i] = sec_base<R>(idx[i], P.rc, j0 + (uint64_t)s * kThreads, i);
#pragma unroll
      for (int kk = 0; kk < MC; ++kk) {
        R U, F;
        const R v = eps_point<R, D, TR, ALPHA>(P, base, kk, U, F);
        const R L = P.eps_b[0] * log_(U) + P.eps_b[1] * log_(F);
        eps_add<R, MC, NE>(acc, nbad, kk, v, L, P, kk < P.m_launch);
      }
#pragma unroll
      for (int i = 0; i < D; ++i) idx[i] = index_step(idx[i], P.gstep[i], n);
      if constexpr (sizeof(R) == 4) {
        if ((s & fold_mask<TR>()) == fold_mask<TR>()) eps_fold<R, MC, NE>(acc);
      }
    }
  }
  eps_epilogue<R, MC, NE>(acc, nbad, P, partial, counters);
}

// Run-time specialised form (FP32, packed shift pairs, POLY from the code
// generator, NE = the plan's orders exactly).  LOG1: the host has shown U > 0
// and F > 0 on the cube and bF = -bU, so L = bU log(U / F) with
// U / F = U (U^2) v0 from values already at hand: one logarithm per value.
// Otherwise L takes both logarithms, and every order counts its own NaN/Inf.
template <int D, int MC, int NE, int TR, int ALPHA, bool LOG1, bool CHECK, class POLY>
__device__ __forceinline__ void eps_body2(const RuleParams<float>& P, double* __restrict__ partial,
                                          unsigned long long* __restrict__ counters, const SampleIO& sio) {
  static_assert(MC % 2 == 0, "shift pairs");
  if (sio.count > 0) {  // single terms: the scalar evaluation
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= sio.count) return;
    const uint64_t j = sio.j[s];
    const int k = sio.k[s];
    uint32_t base[D];
    float z[D];
    float w = 1.0f;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      uint32_t idx = lattice_index(j, P.g[i], P.n);
      base[i] = sec_base<float>(idx, P.rc, j, i);
      if (sio.idx) sio.idx[(size_t)s * D + i] = idx;
      if (sio.coord) sio.coord[(size_t)s * D + i] = sec_coord_used<float>(P, base[i], k, i);
      z[i] = coord_fx<TR, ALPHA>(base[i] + P.shiftx[k][i], P.kor, w);
    }
    float U, F;
    POLY::template eval<D, 1, 2, float>(P, z, U, F);
    float v = recip(U * U * F);
    if constexpr (TR == TR_KOROBOV) v *= korobov_weight_fx(w);
    const float L = P.eps_b[0] * log_(U) + P.eps_b[1] * log_(F);
    for (int o = 0; o < P.eps_orders; ++o) {
      sio.values[(size_t)s * sio.stride + o] = (double)v * P.value_scale;
      v = v * L * P.eps_inv[o];
    }
    return;
  }
  const uint32_t n = (uint32_t)P.n;
  float2 run2[NE][MC / 2];
  Acc<float> acc[NE][MC];
  unsigned nbad[NE];
#pragma unroll
  for (int o = 0; o < NE; ++o) {
    nbad[o] = 0;
#pragma unroll
    for (int p = 0; p < MC / 2; ++p) run2[o][p] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int kk = 0; kk < MC; ++kk) acc[o][kk].init();
  }
  const uint64_t tile_pts = (uint64_t)kThreads * (uint64_t)P.L;
  for (uint64_t tile = blockIdx.x; tile < P.tiles; tile += gridDim.x) {
    const uint64_t j0 = tile * tile_pts + threadIdx.x;
    if (j0 >= P.n) continue;
    uint64_t left = (P.n - j0 + kThreads - 1) / kThreads;
    const int steps = left < (uint64_t)P.L ? (int)left : P.L;
    uint32_t idx[D];
#pragma unroll
    for (int i = 0; i < D; ++i) idx[i] = lattice_index(j0, P.g[i], P.n);
    for (int st = 0; st < steps; ++st) {
      uint32_t base[D];
#pragma unroll
      for (int i = 0; i < D; ++i) base[i] = sec_base<float>(idx[i], P.rc, j0 + (uint64_t)st * kThreads, i);
#pragma unroll
      for (int p = 0; p < MC / 2; ++p) {
        float2 z[D];
        float2 wk = make_float2(1.0f, 1.0f);
#pragma unroll
        for (int i = 0; i < D; ++i)
          z[i] = coord_fx2<TR, ALPHA>(base[i] + P.shiftx[2 * p][i], base[i] + P.shiftx[2 * p + 1][i], P.kor, wk);
        float2 U, Fn;
        POLY::template eval2<D, 1, 2>(P, z, U, Fn);
        const float2 uu = mul2(U, U);
        float2 v = recip_neg2(mul2(uu, Fn));
        float2 L;
        if constexpr (LOG1) {
          const float2 r = mul2(mul2(U, uu), v);  // U / F
          L = make_float2(P.eps_b[0] * log_(r.x), P.eps_b[0] * log_(r.y));
        } else {
          L = make_float2(P.eps_b[0] * log_(U.x) + P.eps_b[1] * log_(-Fn.x),
                          P.eps_b[0] * log_(U.y) + P.eps_b[1] * log_(-Fn.y));
        }
        if constexpr (TR == TR_KOROBOV) v = mul2(v, korobov_weight_fx2(wk));
#pragma unroll
        for (int o = 0; o < NE; ++o) {
          if constexpr (CHECK) {
            const bool oka = finite_(v.x), okb = finite_(v.y);
            nbad[o] += (oka || 2 * p >= P.m_launch) ? 0u : 1u;
            nbad[o] += (okb || 2 * p + 1 >= P.m_launch) ? 0u : 1u;
            run2[o][p] = add2(run2[o][p], make_float2(oka ? v.x : 0.0f, okb ? v.y : 0.0f));
          } else {
            run2[o][p] = add2(run2[o][p], v);
          }
          if (o + 1 < NE) v = mul2(v, mul2(L, make_float2(P.eps_inv[o], P.eps_inv[o])));
        }
      }
#pragma unroll
      for (int i = 0; i < D; ++i) idx[i] = index_step(idx[i], P.gstep[i], n);
      if ((st & fold_mask<TR>()) == fold_mask<TR>()) {
#pragma unroll
        for (int o = 0; o < NE; ++o) {
          unpack_runs<MC>(run2[o], acc[o]);
#pragma unroll
          for (int kk = 0; kk < MC; ++kk) acc[o][kk].fold();
        }
      }
    }
  }
#pragma unroll
  for (int o = 0; o < NE; ++o) unpack_runs<MC>(run2[o], acc[o]);
  eps_epilogue<float, MC, NE>(acc, nbad, P, partial, counters);
}

// Any integer powers, sparse U and F, runtime d and transform: the general
// kernel's evaluation with the orders added (NE = kEpsMax, MC = kEpsAcc / NE).
template <typename R>
__global__ void __launch_bounds__(kThreads)
    general_eps_kernel(const __grid_constant__ GeneralParams<R> G, double* __restrict__ partial,
                       unsigned long long* __restrict__ counters, const SampleIO sio) {
  constexpr int NE = kEpsMax, MC = kEpsAcc / kEpsMax;
  __shared__ R zsh[QMC_DMAX * kThreads];
  const RuleParams<R>& P = G.base;
  if (sio.count > 0) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= sio.count) return;
    R U, F;
    R v = general_eval<R>(G, sio.j[s], sio.k[s], zsh, sio.idx ? sio.idx + (size_t)s * P.d : nullptr,
                          sio.coord ? sio.coord + (size_t)s * P.d : nullptr, U, F);
    const R L = P.eps_b[0] * log_(U) + P.eps_b[1] * log_(F);
    for (int o = 0; o < P.eps_orders; ++o) {
      sio.values[(size_t)s * sio.stride + o] = (double)v * P.value_scale;
      v = v * L * P.eps_inv[o];
    }
    return;
  }
  Acc<R> acc[NE][MC];
#pragma unroll
  for (int o = 0; o < NE; ++o)
#pragma unroll
    for (int kk = 0; kk < MC; ++kk) acc[o][kk].init();
  unsigned nbad[NE];
#pragma unroll
  for (int o = 0; o < NE; ++o) nbad[o] = 0;
  const uint64_t tile_pts = (uint64_t)kThreads * (uint64_t)P.L;
  for (uint64_t tile = blockIdx.x; tile < P.tiles; tile += gridDim.x) {
    const uint64_t j0 = tile * tile_pts + threadIdx.x;
    if (j0 >= P.n) continue;
    uint64_t left = (P.n - j0 + kThreads - 1) / kThreads;
    const int steps = left < (uint64_t)P.L ? (int)left : P.L;
    for (int s = 0; s < steps; ++s) {
      const uint64_t j = j0 + (uint64_t)s * kThreads;
#pragma unroll
      for (int kk = 0; kk < MC; ++kk) {
        if (kk < P.m_launch) {
          R U, F;
          const R v = general_eval<R>(G, j, kk, zsh, nullptr, nullptr, U, F);
          const R L = P.eps_b[0] * log_(U) + P.eps_b[1] * log_(F);
          eps_add<R, MC, NE>(acc, nbad, kk, v, L, P, true);
        }
      }
      if constexpr (sizeof(R) == 4) {
        if ((s & fold_mask_rt(P.tr)) == fold_mask_rt(P.tr)) eps_fold<R, MC, NE>(acc);
      }
    }
  }
  eps_epilogue<R, MC, NE>(acc, nbad, P, partial, counters);
}


// -------------------------------------------- several integrands, one lattice --
//
// SC integrands of one dimension on the same (n, g, shifts, transform): per
// point the lattice indices and bases, per shift pair the triangle
// coordinates are computed once and shared by the SC packed evaluations
// (POLYS::eval2(M, s, ...) gives U_s and -F_s).  Integrand s of this launch is
// integrand s_base + s of the plan; its per-shift CTA slots are group
// s_base + s of [groups][m_total][nblk][2], and its non-finite values are
// counted in counters[2 (s_base + s)] and in the sum's counters[2 count].
template <int D, int MC, int SC, int TR, int ALPHA, bool CHECK, class POLYS>
__device__ __forceinline__ void multi_body(const MultiParams& M, double* __restrict__ partial,
                                           unsigned long long* __restrict__ counters) {
  static_assert(MC % 2 == 0, "shift pairs");
  const RuleParams<float>& P = M.base;
  const uint32_t n = (uint32_t)P.n;
  float2 run2[SC][MC / 2];
  Acc<float> acc[SC][MC];
  unsigned nbad[SC];
  // under Korobov every value is folded on its own: packed on the compensated
  // pairs directly (the same operations as the scalar fold)
  constexpr bool kPackFold = TR == TR_KOROBOV;
  float2 hi2[SC][kPackFold ? MC / 2 : 1], lo2[SC][kPackFold ? MC / 2 : 1];
#pragma unroll
  for (int s = 0; s < SC; ++s)
#pragma unroll
    for (int p = 0; p < (kPackFold ? MC / 2 : 1); ++p) hi2[s][p] = lo2[s][p] = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int s = 0; s < SC; ++s) {
    nbad[s] = 0;
#pragma unroll
    for (int p = 0; p < MC / 2; ++p) run2[s][p] = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int kk = 0; kk < MC; ++kk) acc[s][kk].init();
  }
  const uint64_t tile_pts = (uint64_t)kThreads * (uint64_t)P.L;
  for (uint64_t tile = blockIdx.x; tile < P.tiles; tile += gridDim.x) {
    const uint64_t j0 = tile * tile_pts + threadIdx.x;
    if (j0 >= P.n) continue;
    uint64_t left = (P.n - j0 + kThreads - 1) / kThreads;
    const int steps = left < (uint64_t)P.L ? (int)left : P.L;
    uint32_t idx[D];
#pragma unroll
    for (int i = 0; i < D; ++i) idx[i] = lattice_index(j0, P.g[i], P.n);
    for (int st = 0; st < steps; ++st) {
      uint32_t base[D];
#pragma unroll
      for (int i = 0; i < D; ++i) base[i] = sec_base<float>(idx[i], P.rc, j0 + (uint64_t)st * kThreads, i);
#pragma unroll
      for (int p = 0; p < MC / 2; ++p) {
        float2 z[D];
        float2 wk = make_float2(1.0f, 1.0f);
#pragma unroll
        for (int i = 0; i < D; ++i)
          z[i] = coord_fx2<TR, ALPHA>(base[i] + P.shiftx[2 * p][i], base[i] + P.shiftx[2 * p + 1][i], P.kor, wk);
        float2 w = wk;
        if constexpr (TR == TR_KOROBOV) w = korobov_weight_fx2(w);
#pragma unroll
        for (int s = 0; s < SC; ++s) {
          float2 U, Fn;
          POLYS::eval2(M, s, z, U, Fn);  // s is a constant once the loop is unrolled
          float2 v = recip_neg2(mul2(mul2(U, U), Fn));
          if constexpr (TR == TR_KOROBOV) v = mul2(v, w);
          if constexpr (CHECK) {
            const bool oka = finite_(v.x), okb = finite_(v.y);
            nbad[s] += (oka || 2 * p >= P.m_launch) ? 0u : 1u;
            nbad[s] += (okb || 2 * p + 1 >= P.m_launch) ? 0u : 1u;
            v = make_float2(oka ? v.x : 0.0f, okb ? v.y : 0.0f);
          }
          if constexpr (kPackFold) fast2sum_add2(hi2[s][p], lo2[s][p], v);
          else run2[s][p] = add2(run2[s][p], v);
        }
      }
#pragma unroll
      for (int i = 0; i < D; ++i) idx[i] = index_step(idx[i], P.gstep[i], n);
      if (!kPackFold && (st & fold_mask<TR>()) == fold_mask<TR>()) {
#pragma unroll
        for (int s = 0; s < SC; ++s) {
          unpack_runs<MC>(run2[s], acc[s]);
#pragma unroll
          for (int kk = 0; kk < MC; ++kk) acc[s][kk].fold();
        }
      }
    }
  }
  __shared__ double red[kThreads / 32][SC * MC];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned long long bad_all = 0;
#pragma unroll
  for (int s = 0; s < SC; ++s) {
    if constexpr (kPackFold) {
#pragma unroll
      for (int p = 0; p < MC / 2; ++p) {
        acc[s][2 * p].hi = hi2[s][p].x;
        acc[s][2 * p].lo = lo2[s][p].x;
        acc[s][2 * p + 1].hi = hi2[s][p].y;
        acc[s][2 * p + 1].lo = lo2[s][p].y;
      }
    } else {
      unpack_runs<MC>(run2[s], acc[s]);
    }
#pragma unroll
    for (int kk = 0; kk < MC; ++kk) {
      double t = acc[s][kk].warp_total();
      if (lane == 0) red[warp][s * MC + kk] = t;
    }
    if constexpr (CHECK) {
      unsigned long long bad = warp_sum_u64((unsigned long long)nbad[s]);
      bad_all += bad;
      if (lane == 0 && bad) atomicAdd(&counters[2 * (M.s_base + s)], bad);
    }
  }
  if constexpr (CHECK) {
    if (lane == 0 && bad_all) atomicAdd(&counters[2 * M.count], bad_all);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < SC * MC; t += kThreads) {
    const int s = t / MC, kk = t % MC;
    if (kk >= P.m_launch) continue;
    double acc_s = 0.0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) acc_s += red[w][t];
    const size_t slot = (((size_t)(M.s_base + s) * P.m_total + P.k_base + kk) * P.nblk + blockIdx.x) * 2;
    partial[slot] = acc_s;
    partial[slot + 1] = 0.0;
  }
}

}  // namespace qmc

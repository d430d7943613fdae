// Internal launch descriptors shared by the host launchers and the sm_103a
// kernels.  Everything a kernel needs per launch travels in one struct passed
// as a __grid_constant__ kernel parameter, so the inner loops read shifts and
// polynomial coefficients as constant-bank operands (no shared-memory or
// global loads on the hot path).
#pragma once

#ifdef __CUDACC_RTC__
// run-time compilation (NVRTC): no host headers
typedef unsigned long long uint64_t;
typedef unsigned int uint32_t;
typedef int int32_t;
typedef unsigned char uint8_t;
#else
#include <cstdint>
#endif

#include "../../include/qmc.h"

namespace qmc {

constexpr int kMcMax = 32;      // shifts handled by one launch
constexpr int kDFast = 8;       // largest d with a specialised sector kernel
constexpr int kPolyCoefMax = 168;  // nested-Horner slots: d=8 degree 3 needs 165
constexpr int kTermsMax = 64;   // sparse monomials per polynomial (general kernel)
constexpr int kThreads = 256;   // threads per CTA of the rule kernels
constexpr int kPairCoefMax = 56;  // packed FP32 path: U (deg 1) + F (deg 2) slots at d = 8 is 54
constexpr int kEpsMax = QMC_EPS_MAX;  // epsilon orders of one pass (Eq. 7 expansion)
constexpr int kEpsAcc = 24;     // shifts x orders accumulated by one epsilon launch

enum TransformCode { TR_NONE = 0, TR_BAKER = 1, TR_KOROBOV = 2 };

// Integrand code inside kernels.
enum FKind { FK_CONST = 0, FK_SEPEXP = 1, FK_SECTOR = 2, FK_DEFORMED = 3, FK_TRIG = 4 };

// Number of nested-Horner coefficients of a degree-K polynomial in D variables:
//   K=1: 1 + D; K=2: 1 + D + D(D+1)/2; K=3: adds D(D+1)(D+2)/6.
__host__ __device__ constexpr int poly_slots(int D, int K) {
  return 1 + (K >= 1 ? D : 0) + (K >= 2 ? D * (D + 1) / 2 : 0) + (K >= 3 ? D * (D + 1) * (D + 2) / 6 : 0);
}

// Fixed point: the fractional part of idx/n is held as P = floor(idx 2^64 / n)
// (64-bit), from the 128-bit reciprocal 2^128/n = rhi 2^64 + rlo.
struct Recip {
  uint64_t rhi;
  uint64_t rlo;
};

// Parameters of the per-point rule kernels (single problem).  R = float for
// FP32EVAL, double for FP64.  Shifts are fixed point: u32 (FP32 path, the
// 2^-24 rounding offset of the float conversion folded in) or u64.
template <typename R>
struct RuleParams {
  uint64_t n;
  uint64_t tiles;          // number of point tiles of kThreads * L points
  int32_t L;               // points per thread per tile
  int32_t d;
  int32_t m_launch;        // shifts in this launch (<= kMcMax)
  int32_t k_base;          // global index of this launch's first shift
  int32_t nblk;            // CTAs per shift chunk (partial slots per shift)
  int32_t alpha;           // Korobov weight (transform code TR_KOROBOV)
  int32_t aU, aF;          // integer powers
  int32_t check_finite;    // 1: left out and count NaN/Inf values
  int32_t tr;              // transform code (general kernel)
  R lam;                   // deformation parameter
  double value_scale;      // constant factor of every weighted value (applied in FP64)
  Recip rc;
  uint32_t g[QMC_DMAX];
  uint32_t gstep[QMC_DMAX];     // (kThreads * g_i) mod n
  uint64_t shift64[kMcMax][QMC_DMAX];
  uint32_t shift32[kMcMax][QMC_DMAX];
  uint32_t shiftx[kMcMax][QMC_DMAX];    // FP32 sector path: Delta rounded to 32-bit fixed point
  R kor[8];                // Korobov z(s) = s^(a+1) sum_k kor[k] s^k on s <= 1/2;
                           // kor[7] = (2a+1)!/(a!)^2 (general kernel weight)
  R cU[kPolyCoefMax];      // nested-Horner U (dense kernels)
  R cF[kPolyCoefMax];      // nested-Horner F
  float2 cp[kPairCoefMax];  // packed FP32 path: (c, c) pairs of U's slots, then of -F's
  R sep_c[QMC_DMAX];       // separable: (1 + c z) exp(b z), trig: h as R
  R sep_b[QMC_DMAX];
  // epsilon expansion of Eq. (7): orders f_0..f_{eps_orders-1} of
  // U^(aU + bU eps) F^(aF + bF eps); their CTA slots follow one another
  // ([order][m_total][nblk][2]) and counters[2 o] counts order o's non-finite values
  int32_t eps_orders;
  int32_t m_total;
  R eps_b[2];              // (bU, bF)
  R eps_inv[kEpsMax];      // 1 / k for k = 1..kEpsMax
};

// Shift row k, dimension i, from its 64-bit fixed-point value s64 =
// round(Delta 2^64): the u64 copy (FP64 paths), the 32-bit copy with the
// 2^-24 rounding offset of the 23-bit float conversion folded in (FP32
// separable, general and deformed paths), and the plain 32-bit rounding
// (FP32 sector paths).
template <typename R>
__host__ __device__ inline void set_shift(RuleParams<R>& P, int k, int i, uint64_t s64) {
  P.shift64[k][i] = s64;
  P.shift32[k][i] = (uint32_t)((s64 + 0x80000000ull) >> 32) + 0x100u;
  P.shiftx[k][i] = (uint32_t)((s64 + 0x80000000ull) >> 32);
}

// Scale nested-Horner slots (poly_dense order) by sigma^degree, so that the
// polynomial takes its coordinates divided by sigma.  sigma is a power of
// two, so the scaled evaluation rounds exactly as the unscaled one.
template <typename T>
__host__ __device__ inline void prescale_slots(T* c, int D, int K, double sigma) {
  const double s1 = sigma, s2 = sigma * sigma, s3 = s2 * sigma;
  if (K == 1) {
    for (int i = 0; i < D; ++i) c[1 + i] = (T)((double)c[1 + i] * s1);
    return;
  }
  int off = 1;
  for (int i = 0; i < D; ++i) {
    c[off] = (T)((double)c[off] * s1);
    ++off;
    for (int j = i; j < D; ++j) {
      c[off] = (T)((double)c[off] * s2);
      ++off;
      if (K == 3)
        for (int k = j; k < D; ++k) {
          c[off] = (T)((double)c[off] * s3);
          ++off;
        }
    }
  }
}

// Coordinate scale of the FP32 sector path per transform code (the kernels
// hand U and F the coordinate divided by it): none 2^-32, baker 2^-31,
// Korobov 1 (its z is computed in float from s).
__host__ __device__ inline double fx_sigma(int tr) {
  return tr == TR_NONE ? 0x1p-32 : (tr == TR_BAKER ? 0x1p-31 : 1.0);
}

// Packed FP32 path: (c, c) pairs of U's degree-1 nested-Horner slots, then of
// -F's degree-2 slots (from cU, cF; negation is exact).
template <typename R>
__host__ __device__ inline void fill_pairs(RuleParams<R>& P, int d) {
  const int nu = poly_slots(d, 1), nf = poly_slots(d, 2);
  for (int s = 0; s < nu && s < kPairCoefMax; ++s) P.cp[s] = make_float2((float)P.cU[s], (float)P.cU[s]);
  for (int s = 0; s < nf && nu + s < kPairCoefMax; ++s)
    P.cp[nu + s] = make_float2(-(float)P.cF[s], -(float)P.cF[s]);
}

// Several integrands on one lattice (shared-lattice sweep): the rule's
// parameters plus the (c, c) pairs of each integrand of this launch's chunk.
constexpr int kMultiChunk = 8;  // integrands fused into one launch
struct MultiParams {
  RuleParams<float> base;
  int32_t s_base;   // first integrand of this launch
  int32_t count;    // integrands of the plan (their sum is group `count`)
  float2 cps[kMultiChunk][kPairCoefMax];  // U's then -F's slots, per integrand
};

// Batched sectors in one persistent launch.  A descriptor is one sector's
// rule for one chunk of up to kPersistMc shifts (FP32 packed sector path:
// prescaled dense slots and their (c, c) pairs, shift rows padded with the
// chunk's first row); a work item is (descriptor, j-chunk).  CTAs take items
// from a counter in any order; item q of a sector writes the fixed slots
// [k][q] of that sector, so the result does not depend on the order.
constexpr int kPersistMc = 8;
constexpr int kPjMc = 16;  // shift rows per descriptor of the run-time specialised persistent kernel
struct alignas(16) PersistDesc {
  RuleParams<float> P;
  double* partial;                // the sector's slots [m][nitems][2]
  unsigned long long* counters;   // the sector's counters [2]
  int32_t nitems;                 // j-chunks of the sector
  int32_t pad[3];
};
struct PersistItem {
  uint32_t desc;  // descriptor
  uint32_t item;  // j-chunk of its sector: points [item * chunk, min(n, (item + 1) * chunk))
};
// One descriptor of a persistent launch whose lattices are run-time values
// (the batched ladder walk): its sector's current lattice and result slots.
struct PjLattice {
  uint64_t n;
  uint64_t rhi, rlo;                 // 2^128 / n
  uint32_t g[QMC_DMAX];
  uint32_t gstep[QMC_DMAX];          // (kThreads g_i) mod n
  double* partial;                   // the sector's slots [m][nitems][2]
  unsigned long long* counters;      // the sector's counters
  int32_t nitems;                    // work items of the sector at this lattice
  int32_t pad;
};
struct PersistArgs {
  const PersistDesc* descs;
  const PersistItem* items;
  uint32_t nitems;
  uint32_t chunk;   // points per item, a multiple of kThreads
  unsigned* next;   // item counter, zero at launch
  const PjLattice* lats;  // per descriptor, for kernels with run-time lattices (else null)
};

// Sparse monomial table for the general kernel (any degree, d <= QMC_DMAX).
template <typename R>
struct SparsePoly {
  int32_t nterms;
  int32_t pad;
  R coef[kTermsMax];
  uint8_t expo[kTermsMax][QMC_DMAX];
};

template <typename R>
struct GeneralParams {
  RuleParams<R> base;
  SparsePoly<R> U;
  SparsePoly<R> F;
};

// Sampling mode: the rule kernels evaluate listed (j, k) terms instead of the rule.
struct SampleIO {
  int32_t count;
  int32_t stride;      // epsilon kernels: values per sample (one per order)
  const uint64_t* j;
  const int32_t* k;    // chunk-local shift index
  double* values;      // [count][2] ([count][stride] for the epsilon kernels)
  uint64_t* idx;       // [count][d] or null
  double* coord;       // [count][d] or null
};

// Device workspace layout of one planned rule.
struct Workspace {
  double* partial;               // [m][nblk][2]
  unsigned long long* counters;  // [0] non-finite, [1] deformation violations
  qmc_result* result;            // device copy of the result
  double* per_shift;             // [m][2]
};

}  // namespace qmc

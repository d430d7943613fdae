// Control-variate device code shared by the per-dimension instantiation
// units (cv_inst.cu) and the host driver (cv.cu).
#pragma once

#include "rule_kernels.cuh"

namespace qmc {

constexpr int kCvR = 16;
constexpr int kCvK = 32;
constexpr int kCvDMax = 8;
constexpr int kCvMc = 8;            // shifts per estimator launch
constexpr int kCvTile = 64;         // the pilot is padded to a multiple of 64 points (4 warps x 16)

// Warp-level tensor-core product D = A B + C, A 16x16 (row), B 16x8 (col),
// BF16 operands packed two per 32-bit register, FP32 accumulation.  Lane l
// (group g = l / 4, t = l % 4) holds A[g][2t..2t+1] (a0), A[g+8][2t..] (a1),
// A[g][2t+8..] (a2), A[g+8][2t+8..] (a3); B[2t..2t+1][g] (b0), B[2t+8..][g]
// (b1); D[g][2t..2t+1] (c0, c1) and D[g+8][2t..2t+1] (c2, c3).
__device__ __forceinline__ void mma_bf16_16x8x16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                                 uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// float -> bfloat16 bits, round to nearest even (finite inputs)
__device__ __forceinline__ uint16_t bf16_bits(float v) {
  const uint32_t u = __float_as_uint(v);
  return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}

// ------------------------------------------------------------- estimator --
//
// The rule applied to (f - g)(z(x)) prod_i w(x_i): per point and shift the
// integrand value h = f(z) prod w (the FP32 sector path's fixed-point,
// dithered coordinates) and the surrogate g(z) prod w.
//
// The surrogate is, per dimension, a contraction of 32 Chebyshev values
// T_k(c), c = cos(F pi z_i), against the 16 x 32 parameters a_ri. on tensor
// cores.  A warp takes 32 points at one shift, lane l evaluating point l's
// integrand and its d cosines.  The contraction then runs as TF32 warp MMAs
// m16n8k8 with the 16 ranks as rows (A = the parameters, from shared memory)
// and 8 points as columns (B = the basis), four groups of 8 points per warp.
// Lane (g, t) (g = l / 4, t = l % 4) holds B rows t and t + 4 of every k-step
// of 8: degrees t, t + 4, ..., t + 28 of point g of the group, which it gets
// from the stride-4 Chebyshev recurrence T_{k+4} = 2 T_4 T_k - T_{k-4}
// started at (T_t, T_{4-t}), run on signed values so that it needs no
// negation (the signs are folded into the parameter fragments).
//
// Precision.  The parameters are bfloat16 values, exact in TF32.  Each basis
// value v is split into a TF32 head (v with its low 13 mantissa bits cleared)
// and the exact remainder lo, which goes through a second MMA: whether the
// hardware truncates lo to TF32 or not, a T = a hi + a lo keeps v to within
// 2^-20 |v|.  That error leans toward zero (sign of v, so of T_k) and, like
// the other rounding below, integrates to zero against T_k's equal positive
// and negative measure.  The tensor cores' FP32 accumulation need not round
// to nearest: truncation shrinks every sum toward zero, and on C_ri,
// dominated by its positive constant term, that bias compounds over the d
// factors (measured: 1e-6 of int g at d = 8).  So degree 0 is left out of
// the contraction and a_ri0 added afterwards (round to nearest): the MMA then
// sums only sum_{k>=1} a_rik T_k, which integrates to zero in z_i, and a bias
// proportional to it integrates to zero as well.
//
// Sums.  The estimator needs only sum_points (h - g) and sum_points h, so a
// lane adds the products it holds (16 (rank, point) terms) without gathering
// g per point; it multiplies them by their points' transform weights, which
// are zero for points whose h is not finite and for points past n, so those
// are left out of both sums.

constexpr int kCvWarps = kThreads / 32;

// Warp-level tensor-core product D = A B + C, A 16x8 (row), B 8x8 (col), TF32
// operands (one per 32-bit register), FP32 accumulation.  Lane l (g = l / 4,
// t = l % 4) holds A[g][t] (a0), A[g+8][t] (a1), A[g][t+4] (a2), A[g+8][t+4]
// (a3); B[t][g] (b0), B[t+4][g] (b1); D[g][2t..2t+1] (c0, c1) and
// D[g+8][2t..2t+1] (c2, c3).
__device__ __forceinline__ void mma_tf32_16x8x8(float (&c)[4], const float4& a, float b0, float b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(__float_as_uint(a.x)), "r"(__float_as_uint(a.y)), "r"(__float_as_uint(a.z)), "r"(__float_as_uint(a.w)),
        "r"(__float_as_uint(b0)), "r"(__float_as_uint(b1)));
}

// The same with a zero accumulator (D = A B).
__device__ __forceinline__ void mma_tf32_16x8x8_z(float (&c)[4], const float4& a, float b0, float b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%10,%10,%10,%10};"
      : "=f"(c[0]), "=f"(c[1]), "=f"(c[2]), "=f"(c[3])
      : "r"(__float_as_uint(a.x)), "r"(__float_as_uint(a.y)), "r"(__float_as_uint(a.z)), "r"(__float_as_uint(a.w)),
        "r"(__float_as_uint(b0)), "r"(__float_as_uint(b1)), "f"(0.0f));
}

// Head/remainder split for TF32 operands: hi keeps the sign, exponent and
// top 10 mantissa bits (exact in TF32), lo = v - hi is exact in FP32 (same
// binade) and below 2^-10 |v|.  Inputs are (b0, b1) of two groups packed as
// (group A, group B); the outputs come out per group as the MMA's (b0, b1)
// operand pairs, so no register moves are needed to transpose them.
__device__ __forceinline__ float tf32_head(float v) { return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u); }
__device__ __forceinline__ void split_tf32_t(float2 b0, float2 b1, float2& hA, float2& lA, float2& hB, float2& lB) {
  hA = make_float2(tf32_head(b0.x), tf32_head(b1.x));
  hB = make_float2(tf32_head(b0.y), tf32_head(b1.y));
  lA = make_float2(__fsub_rn(b0.x, hA.x), __fsub_rn(b1.x, hA.y));
  lB = make_float2(__fsub_rn(b0.y, hB.x), __fsub_rn(b1.y, hB.y));
}

struct CvParams {
  RuleParams<float> base;
  float a[kCvR * kCvDMax * kCvK];   // [r][i][k] with row stride d (packed for the actual d)
  float freq;                       // F: 1 -> cos(pi k x), 2 -> cos(2 pi k x)
  float sigma;                      // coordinate scale of the fixed-point path (z = zf sigma)
  int32_t stall_test;               // tcgen05 kernel: 1 = issue no MMA, so every wait runs out (test hook)
};

template <int D, int TR, int ALPHA>
__global__ void __launch_bounds__(kThreads, 2)
    cv_tc_kernel(const __grid_constant__ CvParams C, double* __restrict__ partial,
                 unsigned long long* __restrict__ counters) {
  const RuleParams<float>& P = C.base;
  // A fragments [dimension][k-step][lane]: (a[g][8s+t], a[g+8][8s+t], a[g][8s+t+4], a[g+8][8s+t+4])
  __shared__ float4 afr[D][4][32];
  // cosines of the warp's 32 points, [warp][dimension][pair of groups][g]: (group 2h, group 2h+1)
  __shared__ float2 cbuf[kCvWarps][D][2][8];
  // per point of the warp: its transform weight, 0 for a point left out
  __shared__ __align__(8) float wbuf[kCvWarps][32];
  __shared__ double accs[2][kCvMc][kThreads];
  __shared__ double red[kCvWarps][kCvMc][2];
  // constant terms (a[g][i][0] twice, a[g+8][i][0] twice), added outside the MMA
  __shared__ float4 a0p[D][8];
  for (int q = threadIdx.x; q < D * 4 * 32; q += blockDim.x) {
    const int i = q / 128, s = (q / 32) & 3, l = q & 31, g = l >> 2, t = l & 3;
    const float* ai = C.a + i * kCvK + 8 * s + t;
    const float keep = (s == 0 && t == 0) ? 0.0f : 1.0f;  // degree 0 is not contracted
    const float sg = (s & 1) ? -1.0f : 1.0f;                // the recurrence's sign on k-steps 1 and 3
    afr[i][s][l] = make_float4(sg * keep * ai[g * D * kCvK], sg * keep * ai[(g + 8) * D * kCvK],
                               sg * ai[g * D * kCvK + 4], sg * ai[(g + 8) * D * kCvK + 4]);
  }
  for (int q = threadIdx.x; q < D * 8; q += blockDim.x) {
    const int i = q / 8, g = q % 8;
    const float u = C.a[(g * D + i) * kCvK], v = C.a[((g + 8) * D + i) * kCvK];
    a0p[i][g] = make_float4(u, u, v, v);
  }
  for (int kk = 0; kk < kCvMc; ++kk) {
    accs[0][kk][threadIdx.x] = 0.0;
    accs[1][kk][threadIdx.x] = 0.0;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  // one-hot selectors of the recurrence's start pair (T_t, -T_{4-t}); the
  // second pair's selectors carry the minus sign
  const float e0 = t == 0 ? 1.f : 0.f, e1 = t == 1 ? 1.f : 0.f, e2 = t == 2 ? 1.f : 0.f, e3 = t == 3 ? 1.f : 0.f;
  const float2 s0 = make_float2(e0, e0), s1 = make_float2(e1, e1), s2 = make_float2(e2, e2), s3 = make_float2(e3, e3);
  const float2 n0 = make_float2(-e0, -e0), n1 = make_float2(-e1, -e1), n2 = make_float2(-e2, -e2),
               n3 = make_float2(-e3, -e3);
  const float2 one2 = make_float2(1.0f, 1.0f), m12 = make_float2(-1.0f, -1.0f);
  const uint32_t n = (uint32_t)P.n;
  const int mk = P.m_launch;
  unsigned nbad = 0;
  const uint64_t tile_pts = (uint64_t)kThreads * (uint64_t)P.L;
  for (uint64_t tile = blockIdx.x; tile < P.tiles; tile += gridDim.x) {
    const uint64_t j0 = tile * tile_pts + threadIdx.x;
    const uint64_t jw = tile * tile_pts + (threadIdx.x & ~31u);  // the warp's first point
    if (jw >= P.n) continue;                                        // warp-uniform
    const uint64_t left = (P.n - jw + kThreads - 1) / kThreads;
    const int steps = left < (uint64_t)P.L ? (int)left : P.L;       // warp-uniform trip count
#pragma unroll 1
    for (int kk = 0; kk < mk; ++kk) {
      uint32_t idx[D];
#pragma unroll
      for (int i = 0; i < D; ++i) idx[i] = lattice_index(j0, P.g[i], P.n);
      Acc<float> acv, apl;
      acv.init();
      apl.init();
#pragma unroll 1
      for (int s = 0; s < steps; ++s) {
        const uint64_t j = j0 + (uint64_t)s * kThreads;
        const bool valid = j < P.n;
        // this lane's point: integrand value and the surrogate's cosines
        float zf[D];
        float w = 1.0f;
#pragma unroll
        for (int i = 0; i < D; ++i)
          zf[i] = coord_fx<TR, ALPHA>(base32(frac64(idx[i], P.rc)) + dither32(j, i) + P.shiftx[kk][i], P.kor, w);
        const float U = poly_dense<D, 1>(P.cU, zf);
        const float F = poly_dense<D, 2>(P.cF, zf);
        float h = recip(U * U * F);
        if constexpr (TR == TR_KOROBOV) {
          w = korobov_weight_fx(w);
          h *= w;
        }
        const bool fin = finite_(h);
        const bool ok = valid && fin;
        nbad += (valid && !fin) ? 1u : 0u;
        float* cb = reinterpret_cast<float*>(&cbuf[warp][0][0][0]);
#pragma unroll
        for (int i = 0; i < D; ++i)  // point l = 8 group + g sits at [i][group / 2][g].(group % 2)
          cb[((i * 2 + (lane >> 4)) * 8 + (lane & 7)) * 2 + ((lane >> 3) & 1)] = cospif(C.freq * (zf[i] * C.sigma));
        wbuf[warp][lane] = ok ? w : 0.0f;
        __syncwarp();
        // the surrogate: product over dimensions of the rank values, per (rank,
        // point) held by this lane, for groups 2hp and 2hp + 1 at a time
        float gs = 0.0f;
#pragma unroll 1
        for (int hp = 0; hp < 2; ++hp) {
          float2 prod[2][2];  // [group 2hp + o][rank g / g + 8] x (point 2t, 2t + 1)
          prod[0][0] = prod[0][1] = prod[1][0] = prod[1][1] = one2;
#pragma unroll
          for (int i = 0; i < D; ++i) {
            float4 A[4];
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) A[ks] = afr[i][ks][lane];
            const float2 c = cbuf[warp][i][hp][g];  // point g of groups 2hp, 2hp + 1
            const float2 c2 = add2(c, c);
            const float2 T2 = fma2(c2, c, m12);
            const float2 T3 = fma2(c2, T2, mul2(c, m12));
            const float2 T4 = fma2(add2(T2, T2), T2, m12);
            const float2 two4 = add2(T4, T4), ntwo4 = mul2(T4, make_float2(-2.0f, -2.0f));
            // v_j = s_j T_{t+4j} with signs s = (+, +, -, -, +, +, -, -): then
            // v_{j+1} = (+/-) 2 T_4 v_j + v_{j-1} (+ from even j, - from odd j)
            // needs no negation; v_0 = T_t, v_{-1} = -T_{4-t}
            float2 cur = fma2(s3, T3, fma2(s2, T2, fma2(s1, c, s0)));
            float2 prev = fma2(n3, c, fma2(n2, T2, fma2(n1, T3, mul2(n0, T4))));
            // k-step ks: B rows t, t + 4 = v_{2ks}, v_{2ks+1} (degrees 8 ks + t,
            // 8 ks + t + 4, sign (-1)^ks, undone in A); the recurrence runs on
            // both groups packed (.x, .y), the split hands out each group's
            // (b0, b1) pair
            float chA[4], clA[4], chB[4], clB[4];
#pragma unroll
            for (int ks = 0; ks < 4; ++ks) {
              const float2 b0 = cur;
              const float2 b1 = fma2(two4, cur, prev);
              if (ks < 3) {
                prev = b1;
                cur = fma2(ntwo4, b1, b0);
              }
              float2 hA, lA, hB, lB;
              split_tf32_t(b0, b1, hA, lA, hB, lB);
              if (ks == 0) {
                mma_tf32_16x8x8_z(chA, A[ks], hA.x, hA.y);
                mma_tf32_16x8x8_z(chB, A[ks], hB.x, hB.y);
                mma_tf32_16x8x8_z(clA, A[ks], lA.x, lA.y);
                mma_tf32_16x8x8_z(clB, A[ks], lB.x, lB.y);
              } else {
                mma_tf32_16x8x8(chA, A[ks], hA.x, hA.y);
                mma_tf32_16x8x8(chB, A[ks], hB.x, hB.y);
                mma_tf32_16x8x8(clA, A[ks], lA.x, lA.y);
                mma_tf32_16x8x8(clB, A[ks], lB.x, lB.y);
              }
            }
            // C_ri = a_ri0 + (head + remainder products), rounded to nearest here
            const float4 a0 = a0p[i][g];
            const float2 a0g = make_float2(a0.x, a0.y), a0g8 = make_float2(a0.z, a0.w);
            prod[0][0] = mul2(prod[0][0], add2(add2(make_float2(chA[0], chA[1]), make_float2(clA[0], clA[1])), a0g));
            prod[0][1] = mul2(prod[0][1], add2(add2(make_float2(chA[2], chA[3]), make_float2(clA[2], clA[3])), a0g8));
            prod[1][0] = mul2(prod[1][0], add2(add2(make_float2(chB[0], chB[1]), make_float2(clB[0], clB[1])), a0g));
            prod[1][1] = mul2(prod[1][1], add2(add2(make_float2(chB[2], chB[3]), make_float2(clB[2], clB[3])), a0g8));
          }
#pragma unroll
          for (int o = 0; o < 2; ++o) {  // points 2t, 2t + 1 of group 2hp + o, times their weights
            const float2 wp = *reinterpret_cast<const float2*>(&wbuf[warp][8 * (2 * hp + o) + 2 * t]);
            const float2 gp = mul2(add2(prod[o][0], prod[o][1]), wp);
            gs += gp.x + gp.y;
          }
        }
        __syncwarp();  // cbuf is rewritten by the next step
        const float hv = ok ? h : 0.0f;
        acv.add(hv - gs);
        apl.add(hv);
#pragma unroll
        for (int i = 0; i < D; ++i) idx[i] = index_step(idx[i], P.gstep[i], n);
        if ((s & fold_mask<TR>()) == fold_mask<TR>()) {
          acv.fold();
          apl.fold();
        }
      }
      accs[0][kk][threadIdx.x] += acv.thread_total();
      accs[1][kk][threadIdx.x] += apl.thread_total();
    }
  }
  for (int kk = 0; kk < mk; ++kk) {
    const double a0 = warp_sum_d(accs[0][kk][threadIdx.x]);
    const double a1 = warp_sum_d(accs[1][kk][threadIdx.x]);
    if (lane == 0) {
      red[warp][kk][0] = a0;
      red[warp][kk][1] = a1;
    }
  }
  unsigned long long b1 = warp_sum_u64((unsigned long long)nbad);
  if (lane == 0 && b1) atomicAdd(&counters[0], b1);
  __syncthreads();
  if (threadIdx.x < 2 * mk) {
    const int kk = threadIdx.x >> 1, part = threadIdx.x & 1;
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kCvWarps; ++w) s += red[w][kk][part];
    partial[((size_t)(P.k_base + kk) * P.nblk + blockIdx.x) * 2 + part] = s;
  }
}

// One step of the fit (loss and gradient of the mean squared error) in one
// pass over the pilot points, on tensor cores.  A CTA of kCvFitWarps warps
// takes batches of kCvFitWarps tiles of 16 pilot points (grid-stride over the
// batches).
//
// Forward (warp w on tile w of the batch): per dimension i, C_i = B_i a_i^T
// with the basis tile B_i (16 points x 32 degrees, BF16, Bf[i][j][k]) as A of
// m16n8k16 (two k-steps) and the parameters a[r][i][k] (BF16, shared memory)
// as B (two r-tiles).  A lane holds the same (point, rank) positions of C for
// every dimension, so g = sum_r prod_i C_ri, the error e = 2 (g - h) / P and
// the gradient factor D_i = e prod_{i' != i} C_ri' stay in its registers;
// only the sum over r needs the other three lanes of its group.  The factor
// goes to shared memory as BF16, transposed to D_i^T[r][j] by movmatrix
// (8 x 8 BF16 blocks of the accumulator layout).
//
// Backward (warp w on dimension w, for every tile of the batch):
// grad_w[r][k] += sum_j D_w[j][r] B_w[j][k], four m16n8k16 per tile
// (k-tiles of 8) with A = D_w^T from shared memory and B = the basis tile's
// forward fragments transposed by movmatrix (no transposed basis in memory).
// The gradient of a dimension accumulates in one warp's FP32 registers over
// the CTA's batches, and each CTA writes its partial gradient, which
// cv_adam_kernel sums in FP64 in CTA order.  Rows j >= P (padding) have zero
// basis rows and a zero error, so they add nothing to the loss or gradient.
constexpr int kCvFitWarps = 8;

__device__ __forceinline__ uint32_t movtrans(uint32_t x) {
  uint32_t y;
  asm volatile("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;" : "=r"(y) : "r"(x));
  return y;
}

// two BF16 values in one register, the first in the low half (the lower
// column of an MMA fragment)
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  return (uint32_t)bf16_bits(lo) | ((uint32_t)bf16_bits(hi) << 16);
}

template <int D>
__global__ void __launch_bounds__(kCvFitWarps * 32)
    cv_fit_kernel(const uint16_t* __restrict__ Bf, const double* __restrict__ hv, const float* __restrict__ a, int P,
                  int Ppad, float* __restrict__ grad_part, double* __restrict__ loss_part) {
  constexpr int W = kCvFitWarps;
  static_assert(D <= W, "one warp per dimension in the backward");
  // factors D_i^T of the batch's tiles: [tile][dimension][rank][8 words of 2 points] (BF16
  // pairs); word w of rank row r sits at w ^ (4 ((r >> 2) & 1)), so the eight rows a
  // fragment load touches fall in distinct banks
  __shared__ __align__(16) uint16_t as[kCvR * D * kCvK];
  __shared__ __align__(16) uint32_t fs[W][D][kCvR][8];
  __shared__ double red[W];
  for (int q = threadIdx.x; q < kCvR * D * kCvK; q += blockDim.x) as[q] = bf16_bits(a[q]);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float acc[4][4];  // dimension `warp`: grad[r = g (+8)][k = 8 n + 2t (+1)]
#pragma unroll
  for (int n = 0; n < 4; ++n)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[n][v] = 0.0f;
  double l2 = 0.0;
  const int ntiles = Ppad / 16;
  for (int b0 = blockIdx.x * W; b0 < ntiles; b0 += gridDim.x * W) {
    __syncthreads();  // as[] loaded; fs[] free for this batch
    // ---- forward, warp w on tile b0 + w
    const int tile = b0 + warp;
    if (tile < ntiles) {
      const int j0 = tile * 16;
      float C[D][2][4];  // [dimension][r-tile][fragment]
#pragma unroll
      for (int i = 0; i < D; ++i) {
        const uint16_t* rowA = Bf + ((size_t)i * Ppad + j0 + g) * kCvK;
        const uint16_t* rowB = rowA + 8 * kCvK;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
          for (int v = 0; v < 4; ++v) C[i][nt][v] = 0.0f;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          const int k = 16 * ks + 2 * t;
          const uint32_t a0 = *reinterpret_cast<const uint32_t*>(rowA + k);
          const uint32_t a1 = *reinterpret_cast<const uint32_t*>(rowB + k);
          const uint32_t a2 = *reinterpret_cast<const uint32_t*>(rowA + k + 8);
          const uint32_t a3 = *reinterpret_cast<const uint32_t*>(rowB + k + 8);
#pragma unroll
          for (int nt = 0; nt < 2; ++nt) {
            const uint16_t* ap = as + ((8 * nt + g) * D + i) * kCvK + k;
            const uint32_t b0r = *reinterpret_cast<const uint32_t*>(ap);
            const uint32_t b1r = *reinterpret_cast<const uint32_t*>(ap + 8);
            mma_bf16_16x8x16(C[i][nt], a0, a1, a2, a3, b0r, b1r);
          }
        }
      }
      // g for rows j0 + g (fragments 0, 1) and j0 + g + 8 (fragments 2, 3)
      float gA = 0.0f, gB = 0.0f;
#pragma unroll
      for (int nt = 0; nt < 2; ++nt)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          float p = 1.0f;
#pragma unroll
          for (int i = 0; i < D; ++i) p *= C[i][nt][v];
          if (v < 2) gA += p;
          else gB += p;
        }
      gA += __shfl_xor_sync(0xffffffffu, gA, 1);
      gA += __shfl_xor_sync(0xffffffffu, gA, 2);
      gB += __shfl_xor_sync(0xffffffffu, gB, 1);
      gB += __shfl_xor_sync(0xffffffffu, gB, 2);
      const int jA = j0 + g, jB = j0 + g + 8;
      const double errA = jA < P ? (double)gA - hv[2 * (size_t)jA] : 0.0;
      const double errB = jB < P ? (double)gB - hv[2 * (size_t)jB] : 0.0;
      if (t == 0) l2 += errA * errA + errB * errB;
      const float eA = (float)(2.0 * errA / (double)P), eB = (float)(2.0 * errB / (double)P);
      // D_i in the accumulator layout as BF16 pairs (rows = points g, g + 8;
      // columns = ranks 8 nt + 2t, +1), transposed block by block into
      // D_i^T[r][j]: lane (g, t) then holds ranks 8 nt + g at points 2t, 2t + 1
      // (and 8 + 2t, 9 + 2t)
#pragma unroll
      for (int i = 0; i < D; ++i)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
          float o[4];
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            float p = v < 2 ? eA : eB;
#pragma unroll
            for (int i2 = 0; i2 < D; ++i2)
              if (i2 != i) p *= C[i2][nt][v];
            o[v] = p;
          }
          const int r = 8 * nt + g, sw = 4 * ((r >> 2) & 1);
          fs[warp][i][r][t ^ sw] = movtrans(pack_bf16(o[0], o[1]));
          fs[warp][i][r][(4 + t) ^ sw] = movtrans(pack_bf16(o[2], o[3]));
        }
    }
    __syncthreads();
    // ---- backward, warp w on dimension w, every tile of the batch
    if (warp < D) {
      const int i = warp;
#pragma unroll 1
      for (int b = 0; b < W && b0 + b < ntiles; ++b) {
        const int j0 = (b0 + b) * 16;
        const int sw = 4 * ((g >> 2) & 1);  // rows g and g + 8 share the swizzle
        const uint32_t A0 = fs[b][i][g][t ^ sw];
        const uint32_t A1 = fs[b][i][g + 8][t ^ sw];
        const uint32_t A2 = fs[b][i][g][(4 + t) ^ sw];
        const uint32_t A3 = fs[b][i][g + 8][(4 + t) ^ sw];
        const uint16_t* rowA = Bf + ((size_t)i * Ppad + j0 + g) * kCvK;
        const uint16_t* rowB = rowA + 8 * kCvK;
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          const int k = 16 * ks + 2 * t;
          // the forward's basis fragments, transposed: points 2t.. (first) and
          // 2t + 8.. (second) at degree 16 ks + g (k-tile 2 ks) and 16 ks + 8 + g
          const uint32_t b00 = movtrans(*reinterpret_cast<const uint32_t*>(rowA + k));
          const uint32_t b01 = movtrans(*reinterpret_cast<const uint32_t*>(rowB + k));
          const uint32_t b10 = movtrans(*reinterpret_cast<const uint32_t*>(rowA + k + 8));
          const uint32_t b11 = movtrans(*reinterpret_cast<const uint32_t*>(rowB + k + 8));
          mma_bf16_16x8x16(acc[2 * ks], A0, A1, A2, A3, b00, b01);
          mma_bf16_16x8x16(acc[2 * ks + 1], A0, A1, A2, A3, b10, b11);
        }
      }
    }
  }
  if (warp < D) {
    float* out = grad_part + (size_t)blockIdx.x * (kCvR * D * kCvK);
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      out[(g * D + warp) * kCvK + 8 * n + 2 * t] = acc[n][0];
      out[(g * D + warp) * kCvK + 8 * n + 2 * t + 1] = acc[n][1];
      out[((g + 8) * D + warp) * kCvK + 8 * n + 2 * t] = acc[n][2];
      out[((g + 8) * D + warp) * kCvK + 8 * n + 2 * t + 1] = acc[n][3];
    }
  }
  l2 = warp_sum_d(l2);
  if (lane == 0) red[warp] = l2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int w = 0; w < W; ++w) sum += red[w];
    loss_part[blockIdx.x] = sum;
  }
}

// One explicit specialisation per d, each compiled in its own unit.
template <int D>
const void* cv_estimator_ptr(int tr, int alpha);
template <int D>
const void* cv_estimator5_ptr(int tr, int alpha);  // tcgen05 contraction (cv_tc5.cuh)
template <int D>
const void* cv_fit_ptr();
#define QMC_DECL_CV(D) \
  template <> const void* cv_estimator_ptr<D>(int, int); \
  template <> const void* cv_estimator5_ptr<D>(int, int); \
  template <> const void* cv_fit_ptr<D>();
QMC_DECL_CV(1) QMC_DECL_CV(2) QMC_DECL_CV(3) QMC_DECL_CV(4) QMC_DECL_CV(5) QMC_DECL_CV(6) QMC_DECL_CV(7) QMC_DECL_CV(8)
#undef QMC_DECL_CV

}  // namespace qmc

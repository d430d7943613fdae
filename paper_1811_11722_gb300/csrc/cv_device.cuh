// Control-variate device code shared by the per-dimension instantiation
// units (cv_inst.cu) and the host driver (cv.cu).
#pragma once

#include "rule_kernels.cuh"

namespace qmc {

constexpr int kCvR = 16;
constexpr int kCvK = 32;
constexpr int kCvDMax = 8;
constexpr int kCvMc = 8;            // shifts per estimator launch
constexpr int kCvChunk = 2048;      // pilot points per backward CTA
constexpr int kCvTile = 64;         // pilot points per forward CTA (4 warps x 16); the pilot is padded to it

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

struct CvParams {
  RuleParams<float> base;
  float a[kCvR * kCvDMax * kCvK];   // [r][i][k] with row stride d (packed for the actual d)
  float freq;                       // F: 1 -> cos(pi k x), 2 -> cos(2 pi k x)
  int32_t pad;
};

// ------------------------------------------------------------- estimator --

// sum_r prod_i sum_k a_rik T_k(cos(F pi x_i)) with the Chebyshev recurrence.
template <int D>
__device__ __forceinline__ float cv_g(const CvParams& C, const float* x) {
  float pr[kCvR];
#pragma unroll
  for (int r = 0; r < kCvR; ++r) pr[r] = 1.0f;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const float c1 = cospif(C.freq * x[i]);
    const float two = c1 + c1;
    float cr[kCvR];
#pragma unroll
    for (int r = 0; r < kCvR; ++r) cr[r] = fmaf(C.a[(r * D + i) * kCvK + 1], c1, C.a[(r * D + i) * kCvK]);
    float t0 = 1.0f, t1 = c1;
#pragma unroll
    for (int k = 2; k < kCvK; ++k) {
      const float t2 = fmaf(two, t1, -t0);
#pragma unroll
      for (int r = 0; r < kCvR; ++r) cr[r] = fmaf(C.a[(r * D + i) * kCvK + k], t2, cr[r]);
      t0 = t1;
      t1 = t2;
    }
#pragma unroll
    for (int r = 0; r < kCvR; ++r) pr[r] *= cr[r];
  }
  float g = 0.0f;
#pragma unroll
  for (int r = 0; r < kCvR; ++r) g += pr[r];
  return g;
}

// (h, g) at one point and shift: h = f(z) prod w and g = g(z) prod w, so the
// rule sums (f - g)(z(x)) prod_i w(x_i), which keeps the smoothness and
// periodicity the transform gives f.
template <int D, int TR, int ALPHA>
__device__ __forceinline__ void cv_value(const CvParams& C, const uint32_t* base, int k, float& hv, float& gv) {
  const RuleParams<float>& P = C.base;
  float z[D], x[D];
  float w = 1.0f;
#pragma unroll
  for (int i = 0; i < D; ++i) {
    const uint32_t X = base[i] + P.shift32[k][i];
    x[i] = unit_f32(X) - 1.0f;
    // Korobov factors normalised one by one (exact constant per factor), so
    // h needs no large constant that float could not represent exactly
    z[i] = coord<float, TR, 0>(X, P.kor, P.alpha, w);
  }
  const float U = poly_dense<D, 1>(P.cU, z);
  const float F = poly_dense<D, 2>(P.cF, z);
  float h = recip(U * U * F);
  float gz = cv_g<D>(C, z);  // the surrogate of f, at the transformed point
  if constexpr (TR == TR_KOROBOV) {
    h *= w;
    gz *= w;
  }
  hv = h;
  gv = gz;
}

template <int D, int TR, int ALPHA>
__global__ void __launch_bounds__(kThreads)
    cv_sector_kernel(const __grid_constant__ CvParams C, double* __restrict__ partial,
                     unsigned long long* __restrict__ counters, const SampleIO sio) {
  const RuleParams<float>& P = C.base;
  if (sio.count > 0) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= sio.count) return;
    uint32_t base[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      uint32_t idx = lattice_index(sio.j[s], P.g[i], P.n);
      base[i] = fix_base<float>(idx, P.rc);
      if (sio.idx) sio.idx[(size_t)s * D + i] = idx;
      if (sio.coord) sio.coord[(size_t)s * D + i] = coord_used<float>(base[i] + P.shift32[sio.k[s]][i]);
    }
    float h, g;
    cv_value<D, TR, ALPHA>(C, base, sio.k[s], h, g);
    sio.values[2 * (size_t)s] = (double)h - (double)g;
    sio.values[2 * (size_t)s + 1] = (double)g;
    return;
  }
  __shared__ double accs[2][kCvMc][kThreads];
  const uint32_t n = (uint32_t)P.n;
  const int mk = P.m_launch;
  for (int kk = 0; kk < kCvMc; ++kk) {
    accs[0][kk][threadIdx.x] = 0.0;
    accs[1][kk][threadIdx.x] = 0.0;
  }
  unsigned nbad = 0;
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
      Acc<float> acv, apl;
      acv.init();
      apl.init();
#pragma unroll 1
      for (int s = 0; s < steps; ++s) {
        uint32_t base[D];
#pragma unroll
        for (int i = 0; i < D; ++i) base[i] = fix_base<float>(idx[i], P.rc);
        float h, g;
        cv_value<D, TR, ALPHA>(C, base, kk, h, g);
        float dv = h - g;
        const bool ok = finite_(dv) && finite_(h);
        nbad += ok ? 0u : 1u;
        acv.add(ok ? dv : 0.0f);
        apl.add(ok ? h : 0.0f);
#pragma unroll
        for (int i = 0; i < D; ++i) idx[i] = index_step(idx[i], P.gstep[i], n);
        if ((s & (kFoldG - 1)) == kFoldG - 1) {
          acv.fold();
          apl.fold();
        }
      }
      accs[0][kk][threadIdx.x] += acv.thread_total();
      accs[1][kk][threadIdx.x] += apl.thread_total();
    }
  }
  __shared__ double red[kThreads / 32][kCvMc][2];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
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
    for (int w = 0; w < kThreads / 32; ++w) s += red[w][kk][part];
    partial[((size_t)(P.k_base + kk) * P.nblk + blockIdx.x) * 2 + part] = s;
  }
}

// Forward pass of the fit on tensor cores.  Warp w of the CTA takes pilot
// points j0 .. j0 + 15.  Per dimension i, C_i = Bf_i a_i^T, with the basis
// Bf[i][j][k] (BF16, k contiguous) as A (16 points x 32 k, two k-steps) and
// the parameters a[r][i][k] (BF16, from shared memory) as B (32 k x 16 r,
// two r-tiles).  A lane holds the same (point, r) positions of C for every
// dimension, so the product over dimensions, g = sum_r prod_i C_ri, the loss
// and the gradient factor 2 e prod_{i' != i} C_ri' / P all stay in its
// registers; only the sum over r needs the other three lanes of its group.
// The factor goes out as BF16 in the layout the backward pass reads,
// DgT[i][r][j] (j contiguous).  Rows j >= P (padding) carry zero basis rows,
// add nothing to the loss and get a zero factor.
template <int D>
__global__ void __launch_bounds__(128)
    cv_forward_kernel(const uint16_t* __restrict__ Bf, const double* __restrict__ hv, const float* __restrict__ a,
                      int P, int Ppad, uint16_t* __restrict__ DgT, double* __restrict__ loss_part) {
  __shared__ __align__(16) uint16_t as[kCvR * D * kCvK];
  __shared__ double red[4];
  for (int q = threadIdx.x; q < kCvR * D * kCvK; q += blockDim.x) as[q] = bf16_bits(a[q]);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int j0 = blockIdx.x * kCvTile + warp * 16;
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
        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(ap);
        const uint32_t b1 = *reinterpret_cast<const uint32_t*>(ap + 8);
        mma_bf16_16x8x16(C[i][nt], a0, a1, a2, a3, b0, b1);
      }
    }
  }
  // g for rows j0 + g (fragments 0, 1) and j0 + g + 8 (fragments 2, 3)
  float prod[2][4];
#pragma unroll
  for (int nt = 0; nt < 2; ++nt)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      float p = 1.0f;
#pragma unroll
      for (int i = 0; i < D; ++i) p *= C[i][nt][v];
      prod[nt][v] = p;
    }
  float gA = prod[0][0] + prod[0][1] + prod[1][0] + prod[1][1];
  float gB = prod[0][2] + prod[0][3] + prod[1][2] + prod[1][3];
  gA += __shfl_xor_sync(0xffffffffu, gA, 1);
  gA += __shfl_xor_sync(0xffffffffu, gA, 2);
  gB += __shfl_xor_sync(0xffffffffu, gB, 1);
  gB += __shfl_xor_sync(0xffffffffu, gB, 2);
  const int jA = j0 + g, jB = j0 + g + 8;
  const double errA = jA < P ? (double)gA - hv[2 * (size_t)jA] : 0.0;
  const double errB = jB < P ? (double)gB - hv[2 * (size_t)jB] : 0.0;
  double l2 = t == 0 ? errA * errA + errB * errB : 0.0;
  const float eA = (float)(2.0 * errA / (double)P), eB = (float)(2.0 * errB / (double)P);
  // factor per (dimension, position): e * prefix * suffix over the other dimensions
#pragma unroll
  for (int nt = 0; nt < 2; ++nt)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const float e = v < 2 ? eA : eB;
      const int j = v < 2 ? jA : jB;
      const int r = 8 * nt + 2 * t + (v & 1);
      float pre[D + 1];
      pre[0] = e;
#pragma unroll
      for (int i = 0; i < D; ++i) pre[i + 1] = pre[i] * C[i][nt][v];
      float suf = 1.0f;
#pragma unroll
      for (int i = D - 1; i >= 0; --i) {
        DgT[((size_t)i * kCvR + r) * Ppad + j] = bf16_bits(pre[i] * suf);
        suf *= C[i][nt][v];
      }
    }
  l2 = warp_sum_d(l2);
  if (lane == 0) red[warp] = l2;
  __syncthreads();
  if (threadIdx.x == 0) loss_part[blockIdx.x] = red[0] + red[1] + red[2] + red[3];
}

// One explicit specialisation per d, each compiled in its own unit.
template <int D>
const void* cv_estimator_ptr(int tr, int alpha);
template <int D>
const void* cv_forward_ptr();
#define QMC_DECL_CV(D) \
  template <> const void* cv_estimator_ptr<D>(int, int); \
  template <> const void* cv_forward_ptr<D>();
QMC_DECL_CV(1) QMC_DECL_CV(2) QMC_DECL_CV(3) QMC_DECL_CV(4) QMC_DECL_CV(5) QMC_DECL_CV(6) QMC_DECL_CV(7) QMC_DECL_CV(8)
#undef QMC_DECL_CV

}  // namespace qmc

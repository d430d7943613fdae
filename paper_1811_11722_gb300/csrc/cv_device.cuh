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

template <int D>
__global__ void __launch_bounds__(256)
    cv_forward_kernel(const float* __restrict__ B, const double* __restrict__ hv, const float* __restrict__ a, int P,
                      float* __restrict__ Dg, double* __restrict__ loss_part) {
  __shared__ float as[kCvR * D * kCvK];
  __shared__ double red[8];
  for (int q = threadIdx.x; q < kCvR * D * kCvK; q += blockDim.x) as[q] = a[q];
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  double l2 = 0.0;
  if (j < P) {
    float C[D][kCvR];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      float b[kCvK];
      const float4* bp = reinterpret_cast<const float4*>(B + ((size_t)i * P + j) * kCvK);
#pragma unroll
      for (int q = 0; q < kCvK / 4; ++q) {
        float4 v = bp[q];
        b[4 * q] = v.x;
        b[4 * q + 1] = v.y;
        b[4 * q + 2] = v.z;
        b[4 * q + 3] = v.w;
      }
#pragma unroll
      for (int r = 0; r < kCvR; ++r) {
        float s = 0.0f;
#pragma unroll
        for (int k = 0; k < kCvK; ++k) s = fmaf(as[(r * D + i) * kCvK + k], b[k], s);
        C[i][r] = s;
      }
    }
    float g = 0.0f;
#pragma unroll
    for (int r = 0; r < kCvR; ++r) {
      float p = 1.0f;
#pragma unroll
      for (int i = 0; i < D; ++i) p *= C[i][r];
      g += p;
    }
    const double err = (double)g - hv[2 * (size_t)j];
    l2 = err * err;
    const float e = (float)(2.0 * err / (double)P);
#pragma unroll
    for (int r = 0; r < kCvR; ++r) {
      float pre[D + 1];
      pre[0] = 1.0f;
#pragma unroll
      for (int i = 0; i < D; ++i) pre[i + 1] = pre[i] * C[i][r];
      float suf = 1.0f;
#pragma unroll
      for (int i = D - 1; i >= 0; --i) {
        Dg[((size_t)i * P + j) * kCvR + r] = e * pre[i] * suf;
        suf *= C[i][r];
      }
    }
  }
  l2 = warp_sum_d(l2);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l2;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    loss_part[blockIdx.x] = s;
  }
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

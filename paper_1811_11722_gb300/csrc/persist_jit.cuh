// Run-time specialised persistent batch (device side, compiled by NVRTC).
//
// A descriptor is one sector's rule (Eq. 2) for a chunk of up to kPjMc shifts.
// The host writes, per descriptor, a struct SP whose members are compile-time
// constants of that rule: dimension, transform, n, the 128-bit reciprocal of
// n, g and its per-step increment, the fixed-point shifts, and U and -F as
// straight-line packed code over their nonzero monomials (coefficient pairs
// in a __constant__ array of the descriptor's sector).  pj_sweep<SP> is the
// FP32 packed sector sweep over one work item (a chunk of consecutive j) with
// all of those folded into the instructions: shifts become immediate
// operands of the coordinate adds, coefficients constant-bank operands of the
// packed FMAs.  Its arithmetic is that of the sector kernels' packed path
// (sector_value2 with the sector kernels' coordinates, reciprocal, weight and
// compensated sums), so each value equals theirs bit for bit.
//
// SP provides
//   static constexpr int D, TR, ALPHA, MC (even, <= kPjMc), M (shift rows
//     written back, <= MC), KBASE (first shift of the chunk); bool CHECK
//   static constexpr uint64_t N, RHI, RLO and static uint32_t g(int i),
//     gstep(int i) (not read with run-time lattices)
//   static uint32_t shift(int k, int i)
//   static const float* kor()
//   static void eval2(const float2* z, float2& U, float2& Fn)
#pragma once

#include "rule_kernels.cuh"

namespace qmc {

// RT: the lattice (n, its reciprocal, g, gstep) comes from *lat at run time
// instead of SP's constants (the batched ladder walk moves a descriptor from
// lattice to lattice); everything else stays compiled in, and the arithmetic
// is the same.
template <class SP, bool RT = false>
__device__ __forceinline__ void pj_sweep(uint64_t j0, uint64_t chunk, uint32_t item, int32_t nitems,
                                         double* __restrict__ partial, unsigned long long* __restrict__ counters,
                                         double (*red)[kPjMc], const PjLattice* __restrict__ lat = nullptr) {
  constexpr int D = SP::D, MC = SP::MC, TR = SP::TR, ALPHA = SP::ALPHA;
  static_assert(MC % 2 == 0 && MC <= kPjMc && SP::M <= MC, "shift rows of a descriptor");
  uint64_t N;
  Recip rc;
  uint32_t gg[D], gs[D];
  if constexpr (RT) {
    N = lat->n;
    rc = Recip{lat->rhi, lat->rlo};
#pragma unroll
    for (int i = 0; i < D; ++i) {
      gg[i] = lat->g[i];
      gs[i] = lat->gstep[i];
    }
  } else {
    N = SP::N;
    rc = Recip{SP::RHI, SP::RLO};
#pragma unroll
    for (int i = 0; i < D; ++i) {
      gg[i] = SP::g(i);
      gs[i] = SP::gstep(i);
    }
  }
  const uint64_t j1 = j0 + chunk < N ? j0 + chunk : N;
  Acc<float> acc[MC];
#pragma unroll
  for (int kk = 0; kk < MC; ++kk) acc[kk].init();
  float2 run2[MC / 2];
#pragma unroll
  for (int p = 0; p < MC / 2; ++p) run2[p] = make_float2(0.0f, 0.0f);
  // under Korobov every value is folded on its own: packed on the compensated
  // pairs directly (the same operations as the scalar fold)
  constexpr bool kPackFold = TR == TR_KOROBOV;
  float2 hi2[kPackFold ? MC / 2 : 1], lo2[kPackFold ? MC / 2 : 1];
#pragma unroll
  for (int p = 0; p < (kPackFold ? MC / 2 : 1); ++p) hi2[p] = lo2[p] = make_float2(0.0f, 0.0f);
  unsigned nbad = 0;
  const uint64_t jt = j0 + threadIdx.x;
  if (jt < j1) {
    const int steps = (int)((j1 - jt + kThreads - 1) / kThreads);
    uint32_t idx[D];
#pragma unroll
    for (int i = 0; i < D; ++i) idx[i] = lattice_index(jt, gg[i], N);
    for (int s = 0; s < steps; ++s) {
      uint32_t base[D];
#pragma unroll
      for (int i = 0; i < D; ++i) base[i] = sec_base<float>(idx[i], rc, jt + (uint64_t)s * kThreads, i);
#pragma unroll
      for (int p = 0; p < MC / 2; ++p) {
        float2 z[D];
        float2 w = make_float2(1.0f, 1.0f);
#pragma unroll
        for (int i = 0; i < D; ++i)
          z[i] = coord_fx2<TR, ALPHA>(base[i] + SP::shift(2 * p, i), base[i] + SP::shift(2 * p + 1, i), SP::kor(), w);
        float2 U, Fn;
        SP::eval2(z, U, Fn);
        float2 v = recip_neg2(mul2(mul2(U, U), Fn));
        if constexpr (TR == TR_KOROBOV) v = mul2(v, korobov_weight_fx2(w));
        if constexpr (SP::CHECK) {
          const bool oka = finite_(v.x), okb = finite_(v.y);
          nbad += (oka || 2 * p >= SP::M) ? 0u : 1u;  // padded rows are not counted
          nbad += (okb || 2 * p + 1 >= SP::M) ? 0u : 1u;
          v = make_float2(oka ? v.x : 0.0f, okb ? v.y : 0.0f);
        }
        if constexpr (kPackFold) fast2sum_add2(hi2[p], lo2[p], v);
        else run2[p] = add2(run2[p], v);
      }
#pragma unroll
      for (int i = 0; i < D; ++i) idx[i] = index_step(idx[i], gs[i], (uint32_t)N);
      if (!kPackFold && (s & fold_mask<TR>()) == fold_mask<TR>()) {
        unpack_runs<MC>(run2, acc);
#pragma unroll
        for (int kk = 0; kk < MC; ++kk) acc[kk].fold();
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
  } else {
    unpack_runs<MC>(run2, acc);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int kk = 0; kk < MC; ++kk) {
    const double t = acc[kk].warp_total();
    if (lane == 0) red[warp][kk] = t;
  }
  if constexpr (SP::CHECK) {
    const unsigned long long bad = warp_sum_u64((unsigned long long)nbad);
    if (lane == 0 && bad) atomicAdd(&counters[0], bad);
  }
  __syncthreads();
  if (threadIdx.x < SP::M) {
    double sum = 0.0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) sum += red[w][threadIdx.x];
    const size_t slot = ((size_t)(SP::KBASE + threadIdx.x) * nitems + item) * 2;
    partial[slot] = sum;
    partial[slot + 1] = 0.0;
  }
}

}  // namespace qmc

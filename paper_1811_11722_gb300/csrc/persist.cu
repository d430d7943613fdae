// Batched sectors in one persistent launch: each CTA takes work items
// (sector-and-shift-chunk descriptor, j-chunk) from a global counter, stages
// the descriptor's rule (shifts, coefficient pairs, lattice, transform) into
// shared memory and sweeps the chunk's points for all of its shifts with the
// FP32 packed sector path (sector_value2 reading its coefficients from
// shared memory), the shifts interleaved through registers.  The CTA's
// per-shift sums go to the item's fixed slot, so the final pass (one CTA per
// sector) sees the same layout as a single rule with one slot per j-chunk.
#include "kernel_table.h"
#include "rule_kernels.cuh"

namespace qmc {

static_assert(sizeof(RuleParams<float>) % 16 == 0, "descriptor staging copies 16-byte words");

template <int D, int TR, int ALPHA, bool CHECK>
__device__ __noinline__ void persist_item(const RuleParams<float>& P, uint64_t j0, uint64_t j1, uint32_t item,
                                             int32_t nitems, double* __restrict__ partial,
                                             unsigned long long* __restrict__ counters,
                                             double (*red)[kPersistMc]) {
  constexpr int MC = kPersistMc;
  Acc<float> acc[MC];
#pragma unroll
  for (int kk = 0; kk < MC; ++kk) acc[kk].init();
  float2 run2[MC / 2];
#pragma unroll
  for (int p = 0; p < MC / 2; ++p) run2[p] = make_float2(0.0f, 0.0f);
  // under Korobov every value is folded on its own: packed on the compensated
  // pairs directly, as the specialised kernels do
  constexpr bool kPackFold = TR == TR_KOROBOV;
  float2 hi2[kPackFold ? MC / 2 : 1], lo2[kPackFold ? MC / 2 : 1];
#pragma unroll
  for (int p = 0; p < (kPackFold ? MC / 2 : 1); ++p) hi2[p] = lo2[p] = make_float2(0.0f, 0.0f);
  unsigned nbad = 0;
  const uint64_t jt = j0 + threadIdx.x;
  if (jt < j1) {
    const uint32_t n = (uint32_t)P.n;
    const int steps = (int)((j1 - jt + kThreads - 1) / kThreads);
    uint32_t idx[D];
#pragma unroll
    for (int i = 0; i < D; ++i) idx[i] = lattice_index(jt, P.g[i], P.n);
    for (int s = 0; s < steps; ++s) {
      uint32_t base[D];
#pragma unroll
      for (int i = 0; i < D; ++i) base[i] = sec_base<float>(idx[i], P.rc, jt + (uint64_t)s * kThreads, i);
#pragma unroll
      for (int p = 0; p < MC / 2; ++p) {
        float2 v = sector_value2<D, TR, ALPHA, 1, 2, DensePolys>(P, base, p);
        if constexpr (CHECK) {
          const bool oka = finite_(v.x), okb = finite_(v.y);
          nbad += (oka || 2 * p >= P.m_launch) ? 0u : 1u;  // padded rows are not counted
          nbad += (okb || 2 * p + 1 >= P.m_launch) ? 0u : 1u;
          v = make_float2(oka ? v.x : 0.0f, okb ? v.y : 0.0f);
        }
        if constexpr (kPackFold) fast2sum_add2(hi2[p], lo2[p], v);
        else run2[p] = add2(run2[p], v);
      }
#pragma unroll
      for (int i = 0; i < D; ++i) idx[i] = index_step(idx[i], P.gstep[i], n);
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
  if constexpr (CHECK) {
    const unsigned long long bad = warp_sum_u64((unsigned long long)nbad);
    if (lane == 0 && bad) atomicAdd(&counters[0], bad);
  }
  __syncthreads();
  if (threadIdx.x < P.m_launch) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) s += red[w][threadIdx.x];
    const size_t slot = ((size_t)(P.k_base + threadIdx.x) * nitems + item) * 2;
    partial[slot] = s;
    partial[slot + 1] = 0.0;
  }
}

template <int D>
__device__ __forceinline__ void persist_dispatch_tr(const RuleParams<float>& P, uint64_t j0, uint64_t j1,
                                                    uint32_t item, int32_t nitems, double* partial,
                                                    unsigned long long* counters, double (*red)[kPersistMc]) {
  const bool check = P.check_finite != 0;
  if (P.tr == TR_BAKER) {
    if (check) persist_item<D, TR_BAKER, 0, true>(P, j0, j1, item, nitems, partial, counters, red);
    else persist_item<D, TR_BAKER, 0, false>(P, j0, j1, item, nitems, partial, counters, red);
  } else if (P.tr == TR_KOROBOV) {
    if (check) persist_item<D, TR_KOROBOV, 3, true>(P, j0, j1, item, nitems, partial, counters, red);
    else persist_item<D, TR_KOROBOV, 3, false>(P, j0, j1, item, nitems, partial, counters, red);
  } else {
    if (check) persist_item<D, TR_NONE, 0, true>(P, j0, j1, item, nitems, partial, counters, red);
    else persist_item<D, TR_NONE, 0, false>(P, j0, j1, item, nitems, partial, counters, red);
  }
}

__global__ void __launch_bounds__(kThreads, 1) persist_kernel(const __grid_constant__ PersistArgs A) {
  __shared__ __align__(16) RuleParams<float> P;  // staged with 16-byte stores
  __shared__ double red[kThreads / 32][kPersistMc];
  __shared__ uint32_t cur;
  for (;;) {
    if (threadIdx.x == 0) cur = atomicAdd(A.next, 1u);
    __syncthreads();
    const uint32_t it = cur;
    if (it >= A.nitems) break;  // the same for every thread of the CTA
    const PersistItem wi = A.items[it];
    const PersistDesc* ds = A.descs + wi.desc;
    {
      const int4* src = reinterpret_cast<const int4*>(&ds->P);
      int4* dst = reinterpret_cast<int4*>(&P);
      for (int q = threadIdx.x; q < (int)(sizeof(RuleParams<float>) / 16); q += kThreads) dst[q] = src[q];
    }
    __syncthreads();
    const uint64_t j0 = (uint64_t)wi.item * A.chunk;
    const uint64_t j1 = j0 + A.chunk < P.n ? j0 + A.chunk : P.n;
    double* partial = ds->partial;
    unsigned long long* counters = ds->counters;
    const int32_t nitems = ds->nitems;
    switch (P.d) {
      case 1: persist_dispatch_tr<1>(P, j0, j1, wi.item, nitems, partial, counters, red); break;
      case 2: persist_dispatch_tr<2>(P, j0, j1, wi.item, nitems, partial, counters, red); break;
      case 3: persist_dispatch_tr<3>(P, j0, j1, wi.item, nitems, partial, counters, red); break;
      case 4: persist_dispatch_tr<4>(P, j0, j1, wi.item, nitems, partial, counters, red); break;
      case 5: persist_dispatch_tr<5>(P, j0, j1, wi.item, nitems, partial, counters, red); break;
      case 6: persist_dispatch_tr<6>(P, j0, j1, wi.item, nitems, partial, counters, red); break;
      case 7: persist_dispatch_tr<7>(P, j0, j1, wi.item, nitems, partial, counters, red); break;
      default: persist_dispatch_tr<8>(P, j0, j1, wi.item, nitems, partial, counters, red); break;
    }
    __syncthreads();  // P, red and cur are rewritten for the next item
  }
}

const void* persist_kernel_ptr() { return (const void*)&persist_kernel; }

}  // namespace qmc

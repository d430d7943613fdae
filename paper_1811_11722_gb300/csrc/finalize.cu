// Final deterministic pass of the rule on the GPU: per-shift CTA slots ->
// Q^(k) (Eq. 2), Qbar and the two-pass sigma^2 (Eq. 3).
#include "kernel_table.h"
#include "device_common.cuh"

namespace qmc {

constexpr int kFinThreads = 256;

// One CTA per problem (per group of a problem: the epsilon orders of one
// pass have their slots, counters and results one after another).  Warp w
// adds the CTA slots of (shift, part) tasks w, w+8, ... in a fixed order;
// warp 0 then forms Qbar and the two-pass sigma^2 per part.
__device__ void finalize_one(FinalizeArgs A, int grp, double* q /* shared [m][2] */) {
  const double* all = A.partial;
  const bool sum_group = A.sum_last && grp == A.groups - 1;
  A.partial += (size_t)grp * A.m * A.nblk * 2;
  A.counters += 2 * grp;
  A.result += grp;
  if (A.per_shift) A.per_shift += (size_t)grp * A.m * 2;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int parts = A.is_complex ? 2 : 1;
  const int tasks = A.m * parts;
  const double dn = A.dn;
  for (int t = warp; t < tasks; t += kFinThreads / 32) {
    const int k = t / parts, part = t % parts;
    double s = 0.0;
    if (sum_group) {
      // the sum of the integrands: their slots, group by group in a fixed order
      for (int gg = 0; gg < A.groups - 1; ++gg)
        for (int b = lane; b < A.nblk; b += 32) s += all[(((size_t)gg * A.m + k) * A.nblk + b) * 2 + part];
    } else {
      for (int b = lane; b < A.nblk; b += 32) s += A.partial[((size_t)k * A.nblk + b) * 2 + part];
    }
    s = warp_sum_d(s);
    if (lane == 0) q[2 * k + part] = (s * A.value_scale) / dn + A.offset[part];
  }
  if (!A.is_complex)
    for (int k = threadIdx.x; k < A.m; k += kFinThreads) q[2 * k + 1] = A.offset[1];
  __syncthreads();
  if (A.per_shift)
    for (int t = threadIdx.x; t < 2 * A.m; t += kFinThreads) A.per_shift[t] = q[t];
  if (warp == 0) {
    for (int part = 0; part < 2; ++part) {
      double s = 0.0;
      for (int k = lane; k < A.m; k += 32) s += q[2 * k + part];
      s = warp_sum_d(s);
      const double mean = __shfl_sync(0xffffffffu, s, 0) / (double)A.m;
      double v = 0.0;
      for (int k = lane; k < A.m; k += 32) {
        double dlt = q[2 * k + part] - mean;
        v = fma(dlt, dlt, v);
      }
      v = warp_sum_d(v);
      if (lane == 0) {
        const double var = v / ((double)A.m * (double)(A.m - 1));
        A.result->mean[part] = mean;
        A.result->var[part] = var;
        A.result->err[part] = sqrt(var);
      }
    }
    if (lane == 0) {
      const unsigned long long nf = A.counters[0], dv = A.counters[1];
      A.result->nonfinite = nf;
      A.result->deform_violations = dv;
      A.result->status = nf ? QMC_ENONFINITE : (dv ? QMC_EDEFORM : QMC_OK);
      A.result->reserved = 0;
      A.counters[0] = 0;
      A.counters[1] = 0;
    }
  }
}

__global__ void __launch_bounds__(kFinThreads) finalize_kernel(const FinalizeArgs A) {
  extern __shared__ double q[];
  finalize_one(A, blockIdx.x, q);
}

// Batched final pass: CTA b finalises problem b.
__global__ void __launch_bounds__(kFinThreads) finalize_batch_kernel(const FinalizeArgs* __restrict__ args) {
  extern __shared__ double q[];
  finalize_one(args[blockIdx.x], 0, q);
}

const void* finalize_ptr() { return (const void*)&finalize_kernel; }
const void* finalize_batch_ptr() { return (const void*)&finalize_batch_kernel; }

}  // namespace qmc

// Control-variate estimator with the surrogate's contraction on the fifth-
// generation tensor cores (tcgen05): the basis is written by the threads into
// tensor memory and is the MMA's A operand there, the parameters are the B
// operand in shared memory, and the accumulators are read back from tensor
// memory.
//
// It computes what cv_tc_kernel computes (the rule on (f - g)(z(x)) prod w and
// on f(z(x)) prod w, per shift, FP64 sums): the integrand value h of a point
// and its d cosines c_i = cos(F pi z_i) are identical; the surrogate
//   g = sum_r prod_i (a_ri0 + sum_{k=1..31} a_rik T_k(c_i))
// takes its per-dimension contraction from tcgen05.mma.kind::tf32 instead of
// warp-level mma.sync.
//
// Layout.  The CTA's 256 threads are two groups of 128; group q owns one
// 128-point tile per step, thread t of the group point t, which is row t of the
// MMA (M = 128) and lane t of tensor memory.  Per dimension i:
//   A (tensor memory, 128 lanes x 64 columns): columns 0..31 hold the TF32
//     heads of T_0..T_31 of the lane's point (T_0's column is zero: degree 0
//     stays out of the contraction), columns 32..63 the remainders
//   B (shared memory, K-major, no swizzle): B[k][r] = s a_rik with the sign
//     s = (-1)^floor(k/4) that the basis pairs carry (k >= 1), zero for k = 0,
//     for all d dimensions, written once per CTA
//   D (tensor memory, 32 columns): the head products (ranks 0..15) and the
//     remainder products (ranks 16..31 of the columns), each accumulated over
//     four MMAs of K = 8 (N = 16)
// then C_ri = (head + remainder) + a_ri0 in FP32 round to nearest, the same
// arithmetic as the warp-level kernel, and the lane multiplies its 16 rank
// values across dimensions.
//
// Tensor memory: one allocation of 256 columns per CTA (group q uses columns
// 128 q .. 128 q + 95), so two CTAs fit an SM; the kernel's shared memory
// keeps a third from becoming resident (its allocation would wait).
//
// Synchronisation per (step, dimension) within a group: every thread stores
// its A row (tcgen05.st), waits for the stores, fences, and meets the others
// at a named barrier that also ORs their time-out flags; one thread issues
// the eight MMAs and commits them to the group's mbarrier; every thread waits
// on the mbarrier phase (bounded), fences, and loads its D row.  A wait that
// runs past its bound sets a flag; the barrier's OR makes the whole group
// leave its loop at the next dimension, and the kernel reports the time-out
// in bit 63 of the launch's second counter.
#pragma once

#include "cv_device.cuh"

namespace qmc {

constexpr int kTc5Threads = 256;
constexpr int kTc5Cols = 256;            // tensor-memory columns per CTA
constexpr int kTc5GroupCols = 128;       // per group of 128 threads
constexpr int kTc5AHead = 0, kTc5ARem = 32, kTc5D = 64;
constexpr int kTc5PadBytes = 40 * 1024;  // with the rest (~50 KB): two CTAs fit an SM, three do not
constexpr unsigned long long kTc5TimeoutFlag = 1ull << 63;
constexpr long long kTc5WaitCycles = 4ll << 30;  // about two seconds at 2 GHz

// Instruction descriptor of tcgen05.mma.kind::tf32: D FP32 (bits 4-5 = 1),
// A and B TF32 (bits 7-9, 10-12 = 2), both K-major, N >> 3 in bits 17-22,
// M >> 4 in bits 24-28.  M = 128, N = 16.
constexpr uint32_t kTc5Idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, K-major without swizzle: 16-byte start
// address, leading byte offset (between core matrices adjacent in K) and
// stride byte offset (between 8-row groups), version 1 in bits 46-47.
__device__ __forceinline__ uint64_t tc5_smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

__device__ __forceinline__ void tc5_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc5_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc5_st16(uint32_t taddr, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
      "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
      "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
      : "memory");
}

__device__ __forceinline__ void tc5_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
        "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
        "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
        "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ void tc5_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc5_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// D (tensor memory) = A (tensor memory) B (shared memory), plus D if acc.
__device__ __forceinline__ void tc5_mma(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc, uint32_t acc) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %3, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %4, p;\n"
      "}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b_desc), "r"(acc), "r"(kTc5Idesc)
      : "memory");
}

__device__ __forceinline__ void tc5_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(mbar))
               : "memory");
}

__device__ __forceinline__ bool tc5_try_wait(uint64_t* mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_addr(mbar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase with this parity to complete, at most kTc5WaitCycles;
// false on a time-out.
__device__ __forceinline__ bool tc5_wait(uint64_t* mbar, uint32_t parity) {
  const long long t0 = clock64();
  while (!tc5_try_wait(mbar, parity))
    if (clock64() - t0 > kTc5WaitCycles) return false;
  return true;
}

// Named barrier ID over the 128 threads of a group that ORs a flag.
template <int ID>
__device__ __forceinline__ bool tc5_bar_or(bool flag) {
  uint32_t r;
  asm volatile(
      "{\n"
      ".reg .pred p, q;\n"
      "setp.ne.u32 q, %1, 0;\n"
      "barrier.cta.red.or.pred p, %2, 128, q;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(r)
      : "r"(flag ? 1u : 0u), "n"(ID)
      : "memory");
  return r != 0;
}

template <int D, int TR, int ALPHA>
__global__ void __launch_bounds__(kTc5Threads, 2)
    cv_tc5_kernel(const __grid_constant__ CvParams C, double* __restrict__ partial,
                  unsigned long long* __restrict__ counters) {
  static_assert(kThreads == kTc5Threads, "two groups of 128 threads");
  const RuleParams<float>& P = C.base;
  // B operand: per dimension 16 core matrices of 8 ranks x 4 degrees (128
  // bytes each), core matrix (kb, nb) of dimension i at i * 2048 + kb * 256 +
  // nb * 128 bytes (leading byte offset 256, stride byte offset 128)
  __shared__ __align__(1024) float bsm[D * 512];
  __shared__ float a0s[D][kCvR];
  __shared__ double accs[2][kCvMc][kThreads];
  __shared__ double red[kThreads / 32][kCvMc][2];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_slot;
  __shared__ uint8_t pad[kTc5PadBytes];  // residency: two CTAs per SM (tensor memory)
  if (P.n == 0) static_cast<volatile uint8_t*>(pad)[threadIdx.x] = 0;  // never taken (n >= 2); keeps the reservation

  for (int q = threadIdx.x; q < D * 512; q += kThreads) {
    const int i = q / 512, w = q % 512;
    const int kb = w / 64, nb = (w / 32) & 1, row = (w / 4) & 7, kk = w & 3;
    const int r = nb * 8 + row, k = kb * 4 + kk;
    const float sg = ((k >> 2) & 1) ? -1.0f : 1.0f;  // the basis pairs' sign s_(k/2)
    bsm[q] = k == 0 ? 0.0f : sg * C.a[(r * D + i) * kCvK + k];
  }
  for (int q = threadIdx.x; q < D * kCvR; q += kThreads) {
    const int i = q / kCvR, r = q % kCvR;
    a0s[i][r] = C.a[(r * D + i) * kCvK];
  }
  for (int kk = 0; kk < kCvMc; ++kk) {
    accs[0][kk][threadIdx.x] = 0.0;
    accs[1][kk][threadIdx.x] = 0.0;
  }
  // the parameters were written through the generic proxy; the MMA reads them
  // through the async proxy
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                 "r"((uint32_t)kTc5Cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc5_fence_before();
  __syncthreads();
  tc5_fence_after();

  const int grp = threadIdx.x >> 7, row = threadIdx.x & 127;
  const uint32_t tbase = tmem_slot + (uint32_t)(grp * kTc5GroupCols);
  const uint32_t tlane = tbase + ((uint32_t)((warp & 3) * 32) << 16);  // this warp's 32 lanes
  const bool issuer = row == 0;
  uint32_t phase = 0;
  bool timed_out = false, stop = false;
  unsigned nbad = 0;
  const uint32_t n = (uint32_t)P.n;
  const int mk = P.m_launch;
  const uint64_t tile_pts = (uint64_t)kThreads * (uint64_t)P.L;
  const uint32_t b_base = smem_addr(bsm);
  for (uint64_t tile = blockIdx.x; tile < P.tiles && !stop; tile += gridDim.x) {
    const uint64_t j0 = tile * tile_pts + threadIdx.x;
    const uint64_t jg = tile * tile_pts + (uint64_t)(grp * 128);  // the group's first point
    if (jg >= P.n) continue;                                        // group-uniform
    const uint64_t left = (P.n - jg + kThreads - 1) / kThreads;
    const int steps = left < (uint64_t)P.L ? (int)left : P.L;       // group-uniform trip count
#pragma unroll 1
    for (int kk = 0; kk < mk && !stop; ++kk) {
      uint32_t idx[D];
#pragma unroll
      for (int i = 0; i < D; ++i) idx[i] = lattice_index(j0, P.g[i], P.n);
      Acc<float> acv, apl;
      acv.init();
      apl.init();
#pragma unroll 1
      for (int s = 0; s < steps && !stop; ++s) {
        const uint64_t j = j0 + (uint64_t)s * kThreads;
        const bool valid = j < P.n;
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
        float prod[kCvR];
#pragma unroll
        for (int r = 0; r < kCvR; ++r) prod[r] = 1.0f;
#pragma unroll
        for (int i = 0; i < D; ++i) {
          // basis row of this point, degrees (2u, 2u + 1) as one packed pair
          // Q_u = s_u (T_2u, T_2u+1) with the signs s = (+, +, -, -, +, +, ...):
          // from T_{k+2} = 2 T_2 T_k - T_{k-2} the pairs follow
          // Q_{u+1} = (+/-) 2 T_2 Q_u + Q_{u-1} (+ from even u, - from odd u),
          // one FFMA2 and no negation; s_u sits in the B operand.  Each value
          // is split into its TF32 head and the exact remainder.
          const float c = cospif(C.freq * (zf[i] * C.sigma));
          const float t2 = __fmaf_rn(2.0f * c, c, -1.0f);
          const float2 p2t2 = make_float2(2.0f * t2, 2.0f * t2), m2t2 = make_float2(-2.0f * t2, -2.0f * t2);
          const float2 mone = make_float2(-1.0f, -1.0f);
          float2 qprev = make_float2(1.0f, c);                                  // Q_0
          float2 qcur = make_float2(t2, __fmaf_rn(2.0f * c, t2, -c));           // Q_1
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            float hd[16], rm[16];
#pragma unroll
            for (int u = 0; u < 8; ++u) {  // pair 8 half + u: degrees 16 half + 2u, + 1
              const int pu = 8 * half + u;
              float2 q;
              if (pu == 0) {
                q = make_float2(0.0f, c);  // degree 0: not contracted
              } else if (pu == 1) {
                q = qcur;
              } else {
                q = fma2(((pu - 1) & 1) ? m2t2 : p2t2, qcur, qprev);
                qprev = qcur;
                qcur = q;
              }
              const float2 h2 = make_float2(tf32_head(q.x), tf32_head(q.y));
              const float2 r2 = fma2(h2, mone, q);
              hd[2 * u] = h2.x;
              hd[2 * u + 1] = h2.y;
              rm[2 * u] = r2.x;
              rm[2 * u + 1] = r2.y;
            }
            tc5_st16(tlane + kTc5AHead + 16 * half, hd);
            tc5_st16(tlane + kTc5ARem + 16 * half, rm);
          }
          tc5_wait_st();
          tc5_fence_before();
          if (grp == 0 ? tc5_bar_or<1>(timed_out) : tc5_bar_or<2>(timed_out)) {  // the group leaves together
            stop = true;
            break;
          }
          if (issuer && !C.stall_test) {
            tc5_fence_after();
            const uint32_t bi = b_base + (uint32_t)(i * 2048);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
              tc5_mma(tbase + kTc5D, tbase + kTc5AHead + 8 * ks, tc5_smem_desc(bi + 512 * ks, 256, 128), ks);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
              tc5_mma(tbase + kTc5D + 16, tbase + kTc5ARem + 8 * ks, tc5_smem_desc(bi + 512 * ks, 256, 128), ks);
            tc5_commit(&mbar[grp]);
          }
          if (!tc5_wait(&mbar[grp], phase)) timed_out = true;
          phase ^= 1u;
          tc5_fence_after();
          uint32_t dv[32];
          tc5_ld32(tlane + kTc5D, dv);
          tc5_wait_ld();
#pragma unroll
          for (int r = 0; r < kCvR; r += 2) {
            const float2 hd2 = make_float2(__uint_as_float(dv[r]), __uint_as_float(dv[r + 1]));
            const float2 rm2 = make_float2(__uint_as_float(dv[16 + r]), __uint_as_float(dv[16 + r + 1]));
            const float2 cr = add2(add2(hd2, rm2), make_float2(a0s[i][r], a0s[i][r + 1]));
            const float2 pr = mul2(make_float2(prod[r], prod[r + 1]), cr);
            prod[r] = pr.x;
            prod[r + 1] = pr.y;
          }
        }
        if (stop) break;
        const float wg = ok ? w : 0.0f;
        float gs = 0.0f;
#pragma unroll
        for (int r = 0; r < kCvR; ++r) gs += prod[r];
        gs *= wg;
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
  if (timed_out && issuer) tc5_wait(&mbar[grp], phase ^ 1u);  // MMAs of a commit whose wait ran out
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
  if (timed_out && row == 0) atomicOr(&counters[1], kTc5TimeoutFlag);
  tc5_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc5_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_slot), "r"((uint32_t)kTc5Cols)
                 : "memory");
  }
  if (threadIdx.x < 2 * mk) {
    const int kk = threadIdx.x >> 1, part = threadIdx.x & 1;
    double sm = 0.0;
#pragma unroll
    for (int w2 = 0; w2 < kThreads / 32; ++w2) sm += red[w2][kk][part];
    partial[((size_t)(P.k_base + kk) * P.nblk + blockIdx.x) * 2 + part] = sm;
  }
}

}  // namespace qmc

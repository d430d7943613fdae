// Measured arithmetic peaks of the GPU the library runs on: FP32 and FP64
// fused multiply-add throughput, from kernels of independent dependency chains (8 per thread, enough to cover the
// pipelines' latency) on a full grid, timed with CUDA events.  The roofline
// of the lattice kernels is reported against these as well as against the
// nominal unit count x clock.  Likewise the throughput of the warp-level
// tensor-core instructions the control variate issues (TF32 m16n8k8 in the
// estimator, BF16 m16n8k16 in the fit), 8 independent accumulators per warp:
// the attainable peak of those instructions, below the tcgen05 rate the
// cuBLAS figure measures.
#include <cuda_runtime.h>

#include "plan.h"

namespace qmc {

constexpr int kProbeIters = 4096;
constexpr int kProbeChains = 8;

template <typename R>
__global__ void __launch_bounds__(256) probe_fma_kernel(R seed, R* out) {
  R a[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) a[c] = seed + (R)(threadIdx.x + c);
  const R b = (R)0.999999, d = (R)1e-7;
#pragma unroll 4
  for (int it = 0; it < kProbeIters; ++it) {
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) a[c] = fma(a[c], b, d);
  }
  R s = 0;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s += a[c];
  if (s == (R)-1.2345) out[blockIdx.x] = s;  // keeps the chains live
}

constexpr int kMmaIters = 2048;
constexpr int kMmaChains = 8;

template <bool BF16>
__global__ void __launch_bounds__(256) probe_mma_kernel(float seed, float* out) {
  float c[kMmaChains][4];
#pragma unroll
  for (int q = 0; q < kMmaChains; ++q)
#pragma unroll
    for (int v = 0; v < 4; ++v) c[q][v] = 0.0f;
  const uint32_t a0 = __float_as_uint(seed + (float)threadIdx.x), a1 = __float_as_uint(seed * 0.5f);
  const uint32_t b0 = __float_as_uint(seed * 0.25f), b1 = __float_as_uint(seed * 0.125f);
#pragma unroll 2
  for (int it = 0; it < kMmaIters; ++it) {
#pragma unroll
    for (int q = 0; q < kMmaChains; ++q) {
      if constexpr (BF16)
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(c[q][0]), "+f"(c[q][1]), "+f"(c[q][2]), "+f"(c[q][3])
            : "r"(a0), "r"(a1), "r"(a0), "r"(a1), "r"(b0), "r"(b1));
      else
        asm volatile(
            "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+f"(c[q][0]), "+f"(c[q][1]), "+f"(c[q][2]), "+f"(c[q][3])
            : "r"(a0), "r"(a1), "r"(a0), "r"(a1), "r"(b0), "r"(b1));
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int q = 0; q < kMmaChains; ++q) s += c[q][0] + c[q][1] + c[q][2] + c[q][3];
  if (s == -1.2345f) out[blockIdx.x] = s;  // keeps the accumulators live
}

}  // namespace qmc

using namespace qmc;

extern "C" int qmc_measure_peaks(void* stream, double* out) {
  if (!out) return fail(QMC_EINVAL, "null output");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(QMC_ECUDA, "no CUDA device");
  const int blocks = sms * 8;
  void* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, (size_t)blocks * sizeof(double));
  if (e != cudaSuccess) return cuda_fail(e, "probe buffer");
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  auto timed = [&](auto launch, double work) {
    launch();  // warm-up
    float best = 1e30f;
    for (int rep = 0; rep < 5; ++rep) {
      cudaEventRecord(a, st);
      launch();
      cudaEventRecord(b, st);
      cudaEventSynchronize(b);
      float ms = 0;
      cudaEventElapsedTime(&ms, a, b);
      if (ms < best) best = ms;
    }
    return work / (best * 1e-3);
  };
  const double ops = (double)blocks * 256 * kProbeIters * kProbeChains;
  out[0] = timed([&] { probe_fma_kernel<float><<<blocks, 256, 0, st>>>(1.0f, (float*)buf); }, 2 * ops) / 1e12;
  out[1] = timed([&] { probe_fma_kernel<double><<<blocks, 256, 0, st>>>(1.0, (double*)buf); }, 2 * ops) / 1e12;
  // warp-level MMA: per instruction 2 x 16 x 8 x 8 (TF32) or 2 x 16 x 8 x 16 (BF16) flops
  const double mmas = (double)blocks * (256 / 32) * kMmaIters * kMmaChains;
  out[2] = timed([&] { probe_mma_kernel<false><<<blocks, 256, 0, st>>>(1.0f, (float*)buf); }, 2048.0 * mmas) / 1e12;
  out[3] = timed([&] { probe_mma_kernel<true><<<blocks, 256, 0, st>>>(1.0f, (float*)buf); }, 4096.0 * mmas) / 1e12;
  e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_fail(e, "probe kernels");
  return QMC_OK;
}

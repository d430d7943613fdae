// Measured arithmetic peaks of the GPU the library runs on: FP32 and FP64
// fused multiply-add throughput, from kernels of independent dependency chains (8 per thread, enough to cover the
// pipelines' latency) on a full grid, timed with CUDA events.  The roofline
// of the lattice kernels is reported against these as well as against the
// nominal unit count x clock.
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
  e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(buf);
  if (e != cudaSuccess) return cuda_fail(e, "probe kernels");
  return QMC_OK;
}

// qmc_integrate_noalloc: the single-problem rule for callers that cannot
// allocate device memory (for example code running inside a host callback,
// under an allocator that is locked or exhausted, or embedded in a framework
// that owns every allocation of the process).  It runs the same sector kernel
// and final pass as qmc_integrate, but its scratch (the per-CTA result slots,
// the two counters and the staged result) lives in one file-scope __device__
// array of fixed size instead of memory from cudaMalloc/cudaMallocAsync.
//
// The array exists once per device that loads the library and stays resident
// until the process exits.  Its device address comes from
// cudaGetSymbolAddress, looked up once per device with that device current,
// during the first call made on that device.  Every call shares the array, so
// calls whose work overlaps on the GPU (different streams, or different host
// threads) race on it; callers must order them.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "plan.h"
#include "rule_kernels.cuh"

namespace qmc {

constexpr size_t kNoAllocBytes = 4u << 20;   // 4 MiB of scratch per device
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

static std::mutex g_noalloc_mu;
static void* g_noalloc_addr[kNoAllocMaxDevices];

// Device address of the scratch array on the current device.
static int noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(QMC_EUNSUPPORTED, "device index %d too large", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return QMC_OK;
}

// Coefficients of a term table in the nested-Horner slots of poly_dense,
// written in place (no containers).
template <typename R>
static int pack_dense_into(const qmc_poly& p, int D, int K, R* out) {
  const int slots = poly_slots(D, K);
  for (int s = 0; s < slots; ++s) out[s] = R(0);
  double acc[kPolyCoefMax];
  for (int s = 0; s < slots; ++s) acc[s] = 0.0;
  for (int t = 0; t < p.nterms; ++t) {
    int v[3], nv = 0;
    for (int i = 0; i < D; ++i)
      for (int e = 0; e < p.expo[(size_t)t * D + i]; ++e) {
        if (nv >= 3 || nv >= K) return fail(QMC_EUNSUPPORTED, "term degree above the kernel's");
        v[nv++] = i;
      }
    int slot;
    if (nv == 0) {
      slot = 0;
    } else if (K == 1) {
      slot = 1 + v[0];
    } else {
      // offset of the block of first variable v[0]
      int off = 1;
      for (int a = 0; a < v[0]; ++a) {
        off += 1 + (D - a);
        if (K == 3)
          for (int b = a; b < D; ++b) off += (D - b);
      }
      if (nv == 1) {
        slot = off;
      } else if (K == 2) {
        slot = off + 1 + (v[1] - v[0]);
      } else {
        int o2 = off + 1;
        for (int b = v[0]; b < v[1]; ++b) o2 += 1 + (D - b);
        slot = nv == 2 ? o2 : o2 + 1 + (v[2] - v[1]);
      }
    }
    acc[slot] += p.coef[t];
  }
  for (int s = 0; s < slots; ++s) out[s] = (R)acc[s];
  return QMC_OK;
}

template <typename R>
static int noalloc_run(int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts,
                       const qmc_transform& t, const qmc_integrand* f, qmc_result* out, double* per_shift,
                       cudaStream_t st) {
  RuleParams<R> P;  // on the host stack; passed by value to each launch
  fill_common(P, d, n, g, t, f);
  if (P.tr == TR_KOROBOV && P.alpha != 3)
    return fail(QMC_EUNSUPPORTED, "no-alloc path: Korobov weight 3 only");
  const bool fp32 = sizeof(R) == 4;
  const int mc = fp32 ? (m <= 8 ? 8 : (m <= 16 ? 16 : 32)) : 16;
  const void* func = nullptr;
  switch (d) {
#define QMC_D_CASE(DD) \
  case DD:             \
    func = sector_ptr<R, DD>(mc, P.tr, P.alpha, 1, 2, P.check_finite != 0); \
    break;
    QMC_D_CASE(1) QMC_D_CASE(2) QMC_D_CASE(3) QMC_D_CASE(4) QMC_D_CASE(5) QMC_D_CASE(6) QMC_D_CASE(7)
    QMC_D_CASE(8)
#undef QMC_D_CASE
    default: break;
  }
  if (!func) return fail(QMC_EUNSUPPORTED, "no-alloc path: no sector kernel for this request");
  int rc = pack_dense_into<R>(f->U, d, 1, P.cU);
  if (rc) return rc;
  rc = pack_dense_into<R>(f->F, d, 2, P.cF);
  if (rc) return rc;
  if (fp32) {  // the FP32 kernels hand the polynomials z / fx_sigma (exact powers of two)
    prescale_slots(P.cU, d, 1, fx_sigma(P.tr));
    prescale_slots(P.cF, d, 2, fx_sigma(P.tr));
    fill_pairs(P, d);
  }
  if (P.tr == TR_KOROBOV) {
    double s = 1.0;
    for (int i = 0; i < d; ++i) s *= (double)P.kor[7];
    P.value_scale = s;
  }
  int nblk = 0, L = 0;
  uint64_t tiles = 0;
  rc = choose_grid(func, 0, n, nblk, L, tiles, 0);
  if (rc) return rc;
  // scratch layout: partial [m][nblk][2] | counters [2] | result | per-shift [m][2]
  const size_t partial_bytes = (size_t)m * nblk * 2 * sizeof(double);
  const size_t cnt_off = (partial_bytes + 255) & ~(size_t)255;
  const size_t res_off = cnt_off + 256;
  const size_t ps_off = res_off + ((sizeof(qmc_result) + 255) & ~(size_t)255);
  const size_t need = ps_off + (size_t)m * 2 * sizeof(double);
  if (need > kNoAllocBytes)
    return fail(QMC_EINVAL, "no-alloc path: needs %zu bytes of scratch for m=%d on %d CTAs, the fixed limit is %zu",
                need, m, nblk, kNoAllocBytes);
  void* base = nullptr;
  rc = noalloc_scratch(&base);
  if (rc) return rc;
  char* sc = (char*)base;
  double* partial = (double*)sc;
  unsigned long long* counters = (unsigned long long*)(sc + cnt_off);
  qmc_result* res_stage = (qmc_result*)(sc + res_off);
  double* ps_stage = (double*)(sc + ps_off);
  // the array keeps the previous call's contents: the counters must start at zero
  cudaError_t e = cudaMemsetAsync(counters, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return cuda_fail(e, "clear scratch counters");
  P.L = L;
  P.tiles = tiles;
  P.nblk = nblk;
  SampleIO none;
  std::memset(&none, 0, sizeof(none));
  for (int k0 = 0; k0 < m; k0 += mc) {
    const int mk = m - k0 < mc ? m - k0 : mc;
    P.m_launch = mk;
    P.k_base = k0;
    for (int kk = 0; kk < mc; ++kk)
      for (int i = 0; i < d; ++i) {
        const int src = kk < mk ? k0 + kk : k0;
        const uint64_t s64 = shift_fixed64(shifts[(size_t)src * d + i]);
        set_shift(P, kk, i, s64);
      }
    void* args[4] = {&P, &partial, &counters, &none};
    e = cudaLaunchKernel(func, dim3(nblk), dim3(kThreads), args, 0, st);
    if (e != cudaSuccess) return cuda_fail(e, "no-alloc rule launch");
  }
  const bool out_dev = is_device_pointer(out);
  const bool ps_dev = per_shift ? is_device_pointer(per_shift) : true;
  FinalizeArgs A;
  std::memset(&A, 0, sizeof(A));
  A.partial = partial;
  A.nblk = nblk;
  A.m = m;
  A.is_complex = 0;
  A.dn = (double)n;
  A.value_scale = P.value_scale;
  A.counters = counters;
  A.result = out_dev ? out : res_stage;
  A.per_shift = per_shift ? (ps_dev ? per_shift : ps_stage) : nullptr;
  void* fargs[1] = {&A};
  e = cudaLaunchKernel(finalize_ptr(), dim3(1), dim3(256), fargs, (size_t)m * 2 * sizeof(double), st);
  if (e != cudaSuccess) return cuda_fail(e, "no-alloc final pass");
  if (!out_dev) {
    e = cudaMemcpyAsync(out, res_stage, sizeof(qmc_result), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "no-alloc result copy");
  }
  if (per_shift && !ps_dev) {
    e = cudaMemcpyAsync(per_shift, ps_stage, (size_t)m * 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e, "no-alloc per-shift copy");
  }
  if (!out_dev || (per_shift && !ps_dev)) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "no-alloc synchronise");
    if (!out_dev) return out->status;
  }
  return QMC_OK;
}

}  // namespace qmc

using namespace qmc;

extern "C" int qmc_integrate_noalloc(int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts,
                                     qmc_transform t, const qmc_integrand* f, qmc_result* out, double* per_shift,
                                     void* stream) {
  int rc = validate_problem(d, n, m, g, shifts, t, f);
  if (rc) return rc;
  if (!out) return fail(QMC_EINVAL, "null result pointer");
  if (f->kind != QMC_F_SECTOR || f->aU != -2 || f->aF != -1 || d > kDFast || poly_degree(f->U, d) > 1 ||
      poly_degree(f->F, d) > 2)
    return fail(QMC_EUNSUPPORTED, "no-alloc path: sector U^-2 F^-1 with deg U <= 1, deg F <= 2, d <= %d", kDFast);
  if (f->precision == QMC_FP32EVAL) return noalloc_run<float>(d, n, m, g, shifts, t, f, out, per_shift, (cudaStream_t)stream);
  return noalloc_run<double>(d, n, m, g, shifts, t, f, out, per_shift, (cudaStream_t)stream);
}

// Learned control variate for the lattice rule.
//
// Surrogate (separable rank-R cosine expansion, R = 16, K = 32):
//   g(z) = sum_{r<R} prod_{i<d} C_ri(z_i),  C_ri(z) = sum_{k<K} a_rik cos(F pi k z),
//   int_[0,1]^d g = sum_r prod_i a_ri0          (int_0^1 cos(F pi k z) dz = 0, k >= 1)
// fitted by Adam to the integrand f itself (untransformed variables) on the
// points of a pilot lattice.  The estimator is Q^(k)[f - g] + int g: the rule
// sums (f - g)(z(x)) prod_i w(x_i), and since the substitution z(x) keeps the
// integral, int (g o z) prod w = int g.  Subtracting g before the transform
// keeps the smoothness and periodicity the Korobov transform gives the
// summand; a surrogate fitted to the transformed integrand instead breaks
// them and loses the lattice rule's fast convergence.  The estimator is
// unbiased for any g whose integral is known exactly; the kernel also sums
// the plain Q^(k)[f] in the same pass, so every result carries the plain
// rule's estimate beside the control-variate one and the caller keeps
// whichever has the smaller Eq. (3) error.
//
// Training kernels.  The two contractions of the fit run on tensor cores
// (warp-level BF16 MMA, FP32 accumulation); the loss is summed in FP64:
//   cv_basis     B[i][j][k] = cos(F pi k x_ji) for the pilot points, rounded to
//                BF16, Bf[i][j][k], once per fit; padding points j >= P are zero rows
//   cv_fit       per tile of 16 points: C_ri(x_j) = sum_k B a, g_j,
//                e_j = 2 (g_j - h_j)/P, the factor D[i][j][r] = e_j prod_{i'!=i} C_ri'
//                and grad_part[c][i][r][k] += sum_j D[i][j][r] B[i][j][k], all in
//                registers (cv_device.cuh), one partial gradient per CTA c
//   cv_adam      grad = sum_c grad_part (fixed order), Adam step, cosine-decayed rate
// Each contraction is, per dimension, (points x 32) (32 x 16) forward and
// (16 x points) (points x 32) backward: 16 or 32 output columns.  The
// warp-level MMA keeps a point's 16 values C_ri in the registers of the lanes
// that multiply them across dimensions and differentiate the product, and the
// backward's operands are those registers transposed, so one step reads the
// basis once and nothing else between the contractions goes through memory.
//
// Estimator kernels.  The lattice rule with g subtracted evaluates the
// surrogate's per-dimension contraction on tensor cores too, in TF32 on a
// head/remainder split of each basis value, which keeps FP32 accuracy (a BF16
// basis there would bias Q[f - g] beyond the rule's error): cv_tc5_kernel
// (cv_tc5.cuh) with tcgen05.mma and the basis in tensor memory, or
// cv_tc_kernel (cv_device.cuh) with warp-level mma.sync.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <vector>

#include "cv_device.cuh"
#include "plan.h"

namespace qmc {

// Estimator engine: cv_tc5_kernel (contraction by tcgen05.mma, basis in
// tensor memory; the faster one on GB300) unless QMC_CV_ENGINE=mma, which
// takes cv_tc_kernel (warp-level mma.sync).
static bool cv_engine_tcgen05() {
  const char* e = std::getenv("QMC_CV_ENGINE");
  return !(e && std::strcmp(e, "mma") == 0);
}
// QMC_CV_TEST_STALL=1: the tcgen05 kernel issues no MMA, so its bounded
// waits run out and the call returns QMC_ETIMEOUT (tests the time-out path)
static bool cv_stall_test() {
  const char* e = std::getenv("QMC_CV_TEST_STALL");
  return e && e[0] == '1';
}

// -------------------------------------------------------------- training --

__global__ void cv_iota_kernel(uint64_t* j, int P) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < P) j[t] = (uint64_t)t;
}

__global__ void cv_basis_kernel(const double* __restrict__ x, int P, int Ppad, int d, float freq,
                                uint16_t* __restrict__ Bf) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;  // (i, j)
  if (t >= Ppad * d) return;
  const int i = t / Ppad, j = t % Ppad;
  const double xv = j < P ? x[(size_t)j * d + i] : 0.0;
  uint16_t* out = Bf + ((size_t)i * Ppad + j) * kCvK;
#pragma unroll 4
  for (int k = 0; k < kCvK; ++k)
    out[k] = j < P ? bf16_bits((float)cospi((double)freq * (double)k * xv)) : (uint16_t)0;
}

// Adam step.  A CTA takes 32 parameters: warp w adds the CTAs' partial
// gradients c = w, w + 8, ... in FP64 (coalesced rows of 32), the eight warp
// sums are added in warp order, and warp 0 applies the update.  The order of
// every addition is fixed, so the fit is reproducible.
constexpr int kAdamWarps = 8;
__global__ void __launch_bounds__(kAdamWarps * 32)
    cv_adam_kernel(const float* __restrict__ grad_part, int nchunk, int npar, float* __restrict__ a,
                   float* __restrict__ m1, float* __restrict__ m2, int step, float lr, int band) {
  __shared__ double part[kAdamWarps][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = blockIdx.x * 32 + lane;
  double g = 0.0;
  if (q < npar)
#pragma unroll 4
    for (int c = warp; c < nchunk; c += kAdamWarps) g += (double)grad_part[(size_t)c * npar + q];
  part[warp][lane] = g;
  __syncthreads();
  if (warp != 0 || q >= npar) return;
  if (band > 0 && q % kCvK >= band) {  // a band-limited fit holds the higher degrees at zero
    a[q] = 0.0f;
    return;
  }
  double tot = 0.0;
#pragma unroll
  for (int w = 0; w < kAdamWarps; ++w) tot += part[w][lane];
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float gf = (float)tot;
  const float mm = b1 * m1[q] + (1.0f - b1) * gf;
  const float vv = b2 * m2[q] + (1.0f - b2) * gf * gf;
  m1[q] = mm;
  m2[q] = vv;
  const float mh = mm / (1.0f - powf(b1, (float)step));
  const float vh = vv / (1.0f - powf(b2, (float)step));
  a[q] -= lr * mh / (sqrtf(vh) + eps);
}

static const void* cv_fit_for(int d) {
  switch (d) {
    case 1: return cv_fit_ptr<1>();
    case 2: return cv_fit_ptr<2>();
    case 3: return cv_fit_ptr<3>();
    case 4: return cv_fit_ptr<4>();
    case 5: return cv_fit_ptr<5>();
    case 6: return cv_fit_ptr<6>();
    case 7: return cv_fit_ptr<7>();
    default: return cv_fit_ptr<8>();
  }
}

// CTAs of the fused fit step: two per SM, at most one per batch of
// kCvFitWarps tiles of 16 points.
static int cv_fit_grid(int Ppad) {
  const int sms = device_sms();
  const int batches = (Ppad / 16 + kCvFitWarps - 1) / kCvFitWarps;
  return std::max(1, std::min(batches, 2 * std::max(sms, 1)));
}

// Loss partials into lp[0 .. nchunk) and gradient partials into grad_part[nchunk][npar].
static void cv_fit_step(int d, int P, int Ppad, int nchunk, const uint16_t* Bf, const double* hv, const float* a,
                        float* grad_part, double* lp, cudaStream_t st) {
  void* args[7] = {(void*)&Bf, (void*)&hv, (void*)&a, (void*)&P, (void*)&Ppad, (void*)&grad_part, (void*)&lp};
  cudaLaunchKernel(cv_fit_for(d), dim3(nchunk), dim3(kCvFitWarps * 32), args, 0, st);
}

static float bf16_round(float v) {
  uint32_t u;
  std::memcpy(&u, &v, 4);
  const uint32_t lsb = (u >> 16) & 1u;
  u = (u + 0x7FFFu + lsb) & 0xFFFF0000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

// Device buffers of one fit: pilot coordinates and values, basis, parameters.
struct CvFit {
  int d = 0, P = 0, Ppad = 0, nchunk = 0, npar = 0;
  double* x = nullptr;       // [P][d]
  double* hv = nullptr;      // [P][2] (value, 0)
  uint16_t* Bf = nullptr;    // [d][Ppad][K] BF16
  float* a = nullptr;
  float* m1 = nullptr;
  float* m2 = nullptr;
  float* grad_part = nullptr;
  double* loss_part = nullptr;
  void* block = nullptr;
  ~CvFit() {
    if (block) cudaFree(block);
  }
  int alloc(int d_, int P_) {
    d = d_;
    P = P_;
    Ppad = (P + kCvTile - 1) / kCvTile * kCvTile;
    nchunk = cv_fit_grid(Ppad);
    npar = kCvR * d * kCvK;
    size_t sz[] = {(size_t)P * d * 8,  (size_t)P * 2 * 8,         (size_t)d * Ppad * kCvK * 2,
                   (size_t)npar * 4,   (size_t)npar * 4,          (size_t)npar * 4,
                   (size_t)nchunk * npar * 4, (size_t)nchunk * 8};
    size_t total = 0;
    for (size_t s : sz) total += (s + 255) & ~(size_t)255;
    if (cudaMalloc(&block, total) != cudaSuccess) {
      cudaGetLastError();
      return fail(QMC_ENOMEM, "control-variate fit buffers (%zu bytes)", total);
    }
    char* p = (char*)block;
    void** dst[] = {(void**)&x, (void**)&hv, (void**)&Bf, (void**)&a, (void**)&m1, (void**)&m2,
                    (void**)&grad_part, (void**)&loss_part};
    for (int q = 0; q < 8; ++q) {
      *dst[q] = p;
      p += (sz[q] + 255) & ~(size_t)255;
    }
    return QMC_OK;
  }
};

static double cv_loss_host(const CvFit& F, cudaStream_t st) {
  const int nlp = F.nchunk;
  std::vector<double> lp(nlp);
  cudaMemcpyAsync(lp.data(), F.loss_part, nlp * 8, cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  double s = 0.0;
  for (double v : lp) s += v;
  return s / (double)F.P;
}

static int cv_check(int32_t d, const qmc_cv_config* cfg) {
  if (!cfg) return fail(QMC_EINVAL, "null control-variate config");
  if (cfg->R != kCvR || cfg->K != kCvK)
    return fail(QMC_EUNSUPPORTED, "control variate built for R=%d, K=%d", kCvR, kCvK);
  if (d < 1 || d > kCvDMax) return fail(QMC_EUNSUPPORTED, "control variate needs d <= %d", kCvDMax);
  if (cfg->freq_step != 1 && cfg->freq_step != 2) return fail(QMC_EINVAL, "freq_step must be 1 or 2");
  if (cfg->band < 0 || cfg->band > kCvK) return fail(QMC_EINVAL, "band must be in [0, %d]", kCvK);
  return QMC_OK;
}

}  // namespace qmc

using namespace qmc;

extern "C" {

int qmc_cv_loss_grad(int32_t d, const qmc_cv_config* cfg, int32_t P, const double* x, const double* h,
                     const float* a, double* loss_out, float* grad_out, void* stream) {
  int rc = cv_check(d, cfg);
  if (rc) return rc;
  if (P < 1 || !x || !h || !a || !loss_out || !grad_out) return fail(QMC_EINVAL, "bad loss/gradient arguments");
  cudaStream_t st = (cudaStream_t)stream;
  CvFit F;
  rc = F.alloc(d, P);
  if (rc) return rc;
  std::vector<double> hv(2 * (size_t)P, 0.0);
  for (int j = 0; j < P; ++j) hv[2 * (size_t)j] = h[j];
  cudaMemcpyAsync(F.x, x, (size_t)P * d * 8, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(F.hv, hv.data(), hv.size() * 8, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(F.a, a, (size_t)F.npar * 4, cudaMemcpyHostToDevice, st);
  cv_basis_kernel<<<(F.Ppad * d + 255) / 256, 256, 0, st>>>(F.x, P, F.Ppad, d, (float)cfg->freq_step, F.Bf);
  cv_fit_step(d, P, F.Ppad, F.nchunk, F.Bf, F.hv, F.a, F.grad_part, F.loss_part, st);
  std::vector<float> gp((size_t)F.nchunk * F.npar);
  cudaMemcpyAsync(gp.data(), F.grad_part, gp.size() * 4, cudaMemcpyDeviceToHost, st);
  *loss_out = cv_loss_host(F, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "control-variate gradient");
  for (int q = 0; q < F.npar; ++q) {
    double s = 0.0;
    for (int c = 0; c < F.nchunk; ++c) s += gp[(size_t)c * F.npar + q];
    grad_out[q] = (float)s;
  }
  return QMC_OK;
}

int qmc_cv_train(int32_t d, uint64_t n_pilot, const uint64_t* g_pilot, const double* shift_pilot,
                 qmc_transform t, const qmc_integrand* f, const qmc_cv_config* cfg, float* a_out, double* loss_out,
                 void* stream) {
  int rc = cv_check(d, cfg);
  if (rc) return rc;
  if (!a_out || !shift_pilot) return fail(QMC_EINVAL, "null output or pilot shift");
  if (n_pilot < 64 || n_pilot > (1u << 22)) return fail(QMC_EINVAL, "pilot size must be in [64, 2^22]");
  if (cfg->steps < 1 || cfg->steps > 100000 || !(cfg->lr > 0.0f)) return fail(QMC_EINVAL, "bad steps or lr");
  cudaStream_t st = (cudaStream_t)stream;
  // pilot values h_j and coordinates x_j from the rule's own FP64 kernel (sampling mode)
  std::vector<double> sh2(2 * (size_t)d);
  for (int i = 0; i < d; ++i) sh2[i] = sh2[d + i] = shift_pilot[i];
  qmc_integrand f64 = *f;
  f64.precision = QMC_FP64;
  qmc_transform tnone{QMC_TRANSFORM_NONE, 0};  // g approximates f itself on the cube
  (void)t;
  Plan pilot;
  rc = plan_build(&pilot, d, n_pilot, 2, g_pilot, sh2.data(), tnone, &f64, TuneChoice{});
  if (rc) return rc;
  const int P = (int)n_pilot;
  CvFit F;
  rc = F.alloc(d, P);
  if (rc) return rc;
  uint64_t* dj = nullptr;
  int32_t* dk = nullptr;
  if (cudaMalloc(&dj, (size_t)P * 8) != cudaSuccess || cudaMalloc(&dk, (size_t)P * 4) != cudaSuccess) {
    cudaGetLastError();
    if (dj) cudaFree(dj);
    return fail(QMC_ENOMEM, "pilot index buffers");
  }
  std::unique_ptr<void, void (*)(void*)> g1(dj, [](void* p) { cudaFree(p); });
  std::unique_ptr<void, void (*)(void*)> g2(dk, [](void* p) { cudaFree(p); });
  cv_iota_kernel<<<(P + 255) / 256, 256, 0, st>>>(dj, P);
  cudaMemsetAsync(dk, 0, (size_t)P * 4, st);
  SampleIO sio;
  std::memset(&sio, 0, sizeof(sio));
  sio.count = P;
  sio.j = dj;
  sio.k = dk;
  sio.values = F.hv;
  sio.idx = nullptr;
  sio.coord = F.x;
  {
    const Launch& ln = pilot.launches[0];
    double* partial = nullptr;
    unsigned long long* counters = nullptr;
    void* args[4] = {(void*)ln.params.data(), &partial, &counters, &sio};
    cudaError_t e = cudaLaunchKernel(ln.func, dim3((P + 255) / 256), dim3(kThreads), args, 0, st);
    if (e != cudaSuccess) return cuda_fail(e, "pilot evaluation");
  }
  cv_basis_kernel<<<(F.Ppad * d + 255) / 256, 256, 0, st>>>(F.x, P, F.Ppad, d, (float)cfg->freq_step, F.Bf);
  // pilot mean for the initial constant terms
  std::vector<double> hv(2 * (size_t)P);
  cudaMemcpyAsync(hv.data(), F.hv, hv.size() * 8, cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "pilot");
  double qp = 0.0;
  for (int j = 0; j < P; ++j) qp += hv[2 * (size_t)j];
  qp /= (double)P;
  // initialisation: a_ri0 = (Q_pilot / R)^(1/d) (sign kept on r = 0), others N(0, 1e-3) (SplitMix64 + Box-Muller)
  std::vector<float> a0(F.npar);
  uint64_t state = cfg->seed;
  auto next = [&]() {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  auto unif = [&]() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); };
  const double c0 = std::pow(std::fabs(qp) / kCvR, 1.0 / d);
  for (int r = 0; r < kCvR; ++r)
    for (int i = 0; i < d; ++i)
      for (int k = 0; k < kCvK; ++k) {
        const double u1 = unif(), u2 = unif();
        const double nrm = std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
        double v = 1e-3 * nrm;
        if (k == 0) v = c0 * ((qp < 0 && i == 0) ? -1.0 : 1.0) + 1e-3 * nrm;
        if (cfg->band > 0 && k >= cfg->band) v = 0.0;
        a0[(r * d + i) * kCvK + k] = (float)v;
      }
  cudaMemcpyAsync(F.a, a0.data(), (size_t)F.npar * 4, cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(F.m1, 0, (size_t)F.npar * 4, st);
  cudaMemsetAsync(F.m2, 0, (size_t)F.npar * 4, st);
  double first = 0.0, last = 0.0;
  for (int step = 1; step <= cfg->steps; ++step) {
    cv_fit_step(d, P, F.Ppad, F.nchunk, F.Bf, F.hv, F.a, F.grad_part, F.loss_part, st);
    if (step == 1) first = cv_loss_host(F, st);
    const float lr = (float)(0.5 * cfg->lr * (1.0 + std::cos(M_PI * (double)(step - 1) / (double)cfg->steps)));
    cv_adam_kernel<<<(F.npar + 31) / 32, kAdamWarps * 32, 0, st>>>(F.grad_part, F.nchunk, F.npar, F.a, F.m1, F.m2,
                                                                  step, lr, cfg->band);
  }
  cv_fit_step(d, P, F.Ppad, F.nchunk, F.Bf, F.hv, F.a, F.grad_part, F.loss_part, st);
  last = cv_loss_host(F, st);
  std::vector<float> af(F.npar);
  cudaMemcpyAsync(af.data(), F.a, (size_t)F.npar * 4, cudaMemcpyDeviceToHost, st);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "control-variate training");
  for (int q = 0; q < F.npar; ++q) a_out[q] = bf16_round(af[q]);
  if (loss_out) {
    loss_out[0] = first;
    loss_out[1] = last;
  }
  return QMC_OK;
}

int qmc_integrate_cv(int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts, qmc_transform t,
                     const qmc_integrand* f, const qmc_cv_config* cfg, const float* a, qmc_result* out,
                     double* per_shift, void* stream) {
  int rc = cv_check(d, cfg);
  if (rc) return rc;
  rc = validate_problem(d, n, m, g, shifts, t, f);
  if (rc) return rc;
  if (!a || !out) return fail(QMC_EINVAL, "null parameters or result");
  if (f->kind != QMC_F_SECTOR || f->precision != QMC_FP32EVAL || f->aU != -2 || f->aF != -1 ||
      poly_degree(f->U, d) > 1 || poly_degree(f->F, d) > 2)
    return fail(QMC_EUNSUPPORTED, "control variate: FP32EVAL U^-2 F^-1 sector with deg U <= 1, deg F <= 2");
  const int tr = t.kind == QMC_TRANSFORM_KOROBOV ? TR_KOROBOV : (t.kind == QMC_TRANSFORM_BAKER ? TR_BAKER : TR_NONE);
  const bool tc5 = cv_engine_tcgen05();
  const void* func = nullptr;
  switch (d) {
#define QMC_CV_CASE(DD) \
  case DD:             \
    func = tc5 ? cv_estimator5_ptr<DD>(tr, t.alpha) : cv_estimator_ptr<DD>(tr, t.alpha); \
    break;
    QMC_CV_CASE(1) QMC_CV_CASE(2) QMC_CV_CASE(3) QMC_CV_CASE(4) QMC_CV_CASE(5) QMC_CV_CASE(6) QMC_CV_CASE(7)
    QMC_CV_CASE(8)
#undef QMC_CV_CASE
  }
  if (!func) return fail(QMC_EUNSUPPORTED, "control variate: transform must be none, baker or Korobov 3");
  std::unique_ptr<CvParams> C(new CvParams());
  std::memset(C.get(), 0, sizeof(CvParams));
  fill_common(C->base, d, n, g, t, f);
  // the integrand on the FP32 sector path's fixed-point coordinates: U and F
  // take z / fx_sigma (exact powers of two folded into the coefficients)
  auto cu = pack_dense(f->U, d, 1);
  auto cf = pack_dense(f->F, d, 2);
  prescale_slots(cu.data(), d, 1, fx_sigma(C->base.tr));
  prescale_slots(cf.data(), d, 2, fx_sigma(C->base.tr));
  for (size_t i = 0; i < cu.size(); ++i) C->base.cU[i] = (float)cu[i];
  for (size_t i = 0; i < cf.size(); ++i) C->base.cF[i] = (float)cf[i];
  C->base.value_scale = 1.0;
  C->sigma = (float)fx_sigma(C->base.tr);
  const int npar = kCvR * d * kCvK;
  for (int q = 0; q < npar; ++q) C->a[q] = a[q];
  C->freq = (float)cfg->freq_step;
  C->stall_test = tc5 && cv_stall_test() ? 1 : 0;
  double gint = 0.0;
  for (int r = 0; r < kCvR; ++r) {
    double p = 1.0;
    for (int i = 0; i < d; ++i) p *= (double)a[(r * d + i) * kCvK];
    gint += p;
  }
  Plan pl;
  pl.d = d;
  pl.n = n;
  pl.m = m;
  pl.is_complex = 1;
  // Korobov weights go in unnormalised (u^3 per factor); their constant
  // (2a+1)!/(a!)^2 per dimension is applied to both sums in FP64, before int g
  // is added
  pl.final_scale = C->base.tr == TR_KOROBOV ? std::pow((double)C->base.kor[7], (double)d) : 1.0;
  pl.offset[0] = gint;
  pl.mc = kCvMc;
  int nblk = 0, L = 0;
  uint64_t tiles = 0;
  // the tcgen05 kernel is built for two resident CTAs per SM (its tensor
  // memory and shared memory admit two, not three)
  rc = tc5 ? grid_shape(2, n, 0, 0, nblk, L, tiles) : choose_grid(func, 0, n, nblk, L, tiles, 0);
  if (rc) return rc;
  C->base.L = L;
  C->base.tiles = tiles;
  C->base.nblk = nblk;
  pl.nblk = nblk;
  pl.func = func;
  for (int k0 = 0; k0 < m; k0 += kCvMc) {
    const int mk = std::min(kCvMc, m - k0);
    C->base.m_launch = mk;
    C->base.k_base = k0;
    for (int kk = 0; kk < kCvMc; ++kk)
      for (int i = 0; i < d; ++i) {
        const int src = kk < mk ? k0 + kk : k0;
        uint64_t s64 = shift_fixed64(shifts[(size_t)src * d + i]);
        set_shift(C->base, kk, i, s64);
      }
    Launch ln;
    ln.func = func;
    ln.grid = dim3(nblk);
    ln.params.resize(sizeof(CvParams));
    std::memcpy(ln.params.data(), C.get(), sizeof(CvParams));
    pl.launches.push_back(std::move(ln));
  }
  cudaStream_t st = (cudaStream_t)stream;
  rc = plan_alloc(&pl, st, true);
  if (rc) return rc;
  rc = plan_execute(&pl, out, per_shift, st);
  plan_free(&pl, st);
  // the tcgen05 kernel reports a bounded wait that ran out in bit 63 of the
  // second counter (no deformation in these plans)
  if (tc5 && !is_device_pointer(out) && (out->deform_violations & (1ull << 63))) {
    out->status = QMC_ETIMEOUT;
    return fail(QMC_ETIMEOUT, "control variate: a tensor-core wait timed out");
  }
  return rc;
}

// Automatic choice of n with the control variate as a candidate, judged on
// the first lattices (the pilot) by predicted time to the tolerance.
int qmc_integrate_cv_to_tolerance(int32_t d, int32_t levels, const uint64_t* n, const uint64_t* g, int32_t m,
                                  const double* shifts, qmc_transform t, const qmc_integrand* f,
                                  const qmc_cv_config* cfg, const float* a, double rel_tol, qmc_result* out,
                                  int32_t* level_out, int32_t* mode_out, double* judge_out, void* stream) {
  if (levels < 1 || levels > 64 || !n || !g || !out || !a || !(rel_tol > 0.0))
    return fail(QMC_EINVAL, "bad ladder arguments");
  if (is_device_pointer(out)) return fail(QMC_EINVAL, "the result must be host memory");
  using clock = std::chrono::steady_clock;
  auto rel = [](const qmc_result& r, int part) {
    const double mag = std::fabs(r.mean[part]);
    return mag > 0.0 ? r.err[part] / mag : HUGE_VAL;
  };
  auto take_cv = [&](const qmc_result& r) {
    std::memset(out, 0, sizeof(*out));
    out->mean[0] = r.mean[0];
    out->var[0] = r.var[0];
    out->err[0] = r.err[0];
    out->nonfinite = r.nonfinite;
    out->status = r.status;
  };
  // pilot: on each of the first lattices a control-variate pass (Q[f - g] + int g
  // in part 0) and a plain pass (qmc_integrate, so the plain walk is exactly
  // qmc_integrate_to_tolerance's), both run once more at the first lattice so
  // that first-use work (run-time compilation, module loading) stays out of the
  // times; the passes on the last pilot lattice are timed
  const int pilot = std::min(levels, 3);
  std::vector<double> lr(pilot), ecv(pilot), epl(pilot);
  double t_cv = 0.0, t_plain = 0.0;
  int rc = QMC_OK;
  for (int l = 0; l < pilot; ++l) {
    const uint64_t* gl = g + (size_t)l * d;
    qmc_result rcv, rpl;
    for (int rep = 0; rep < (l == 0 ? 2 : 1); ++rep) {
      auto t0 = clock::now();
      rc = qmc_integrate_cv(d, n[l], m, gl, shifts, t, f, cfg, a, &rcv, nullptr, stream);
      if (rc != QMC_OK && rc != QMC_ENONFINITE) return rc;
      auto t1 = clock::now();
      rc = qmc_integrate(d, n[l], m, gl, shifts, t, f, &rpl, nullptr, stream);
      if (rc != QMC_OK && rc != QMC_ENONFINITE) return rc;
      auto t2 = clock::now();
      t_cv = std::chrono::duration<double>(t1 - t0).count();
      t_plain = std::chrono::duration<double>(t2 - t1).count();
    }
    lr[l] = std::log((double)n[l]);
    ecv[l] = rel(rcv, 0);
    epl[l] = rel(rpl, 0);
    if (level_out) *level_out = l;
    if (epl[l] <= rel_tol) {
      *out = rpl;
      if (mode_out) *mode_out = 0;
      return out->status;
    }
    if (ecv[l] <= rel_tol) {
      take_cv(rcv);
      if (mode_out) *mode_out = 1;
      return out->status;
    }
    if (l == pilot - 1) *out = rpl;
  }
  // convergence rate p of each estimate, err ~ n^-p: least-squares slope of
  // log err against log n over the pilot (p = 1 with a single lattice),
  // clamped to [1/4, 8]; predicted time to rel_tol = time per pass on the last
  // pilot lattice x the growth of n it needs, (err / rel_tol)^(1/p)
  auto rate = [&](const std::vector<double>& e) {
    if (pilot < 2) return 1.0;
    double mx = 0.0, my = 0.0;
    for (int l = 0; l < pilot; ++l) {
      mx += lr[l];
      my += std::log(e[l]);
    }
    mx /= pilot;
    my /= pilot;
    double sxy = 0.0, sxx = 0.0;
    for (int l = 0; l < pilot; ++l) {
      sxy += (lr[l] - mx) * (std::log(e[l]) - my);
      sxx += (lr[l] - mx) * (lr[l] - mx);
    }
    const double p = sxx > 0.0 ? -sxy / sxx : 1.0;
    return std::min(8.0, std::max(0.25, std::isfinite(p) ? p : 1.0));
  };
  const double p_cv = rate(ecv), p_plain = rate(epl);
  const int lp = pilot - 1;
  const double T_cv = t_cv * std::pow(std::max(1.0, ecv[lp] / rel_tol), 1.0 / p_cv);
  const double T_plain = t_plain * std::pow(std::max(1.0, epl[lp] / rel_tol), 1.0 / p_plain);
  const bool keep_cv = T_cv < T_plain;
  if (judge_out) {
    const double j[8] = {ecv[lp], epl[lp], t_cv, t_plain, p_cv, p_plain, T_cv, T_plain};
    std::memcpy(judge_out, j, sizeof(j));
  }
  if (mode_out) *mode_out = keep_cv ? 1 : 0;
  for (int l = pilot; l < levels; ++l) {
    const uint64_t* gl = g + (size_t)l * d;
    if (level_out) *level_out = l;
    if (keep_cv) {
      qmc_result r;
      rc = qmc_integrate_cv(d, n[l], m, gl, shifts, t, f, cfg, a, &r, nullptr, stream);
      if (rc != QMC_OK && rc != QMC_ENONFINITE) return rc;
      take_cv(r);
      if (rel(r, 0) <= rel_tol) return out->status;
    } else {
      rc = qmc_integrate(d, n[l], m, gl, shifts, t, f, out, nullptr, stream);
      if (rc != QMC_OK && rc != QMC_ENONFINITE) return rc;
      if (rel(*out, 0) <= rel_tol) return out->status;
    }
  }
  out->status = QMC_ETIMEOUT;
  return fail(QMC_ETIMEOUT, "relative error %.3g not reached after %d lattices", rel_tol, levels);
}

}  // extern "C"

// C ABI of the lattice-rule library: argument validation, packing of the
// problem into launch descriptors, plans, kernel dispatch and the final pass.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstddef>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "kernel_table.h"
#include "plan.h"

namespace qmc {

// ------------------------------------------------------------------ errors --

static thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(QMC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define QMC_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

bool is_device_pointer(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ------------------------------------------------------------- validation --

static bool is_prime_u64(uint64_t n) {
  if (n < 2) return false;
  for (uint64_t p : {2ull, 3ull, 5ull, 7ull, 11ull, 13ull, 17ull, 19ull, 23ull, 29ull, 31ull, 37ull}) {
    if (n % p == 0) return n == p;
  }
  uint64_t d = n - 1;
  int s = 0;
  while ((d & 1) == 0) {
    d >>= 1;
    ++s;
  }
  auto mulmod = [&](uint64_t a, uint64_t b) { return (uint64_t)((unsigned __int128)a * b % n); };
  auto powmod = [&](uint64_t a, uint64_t e) {
    uint64_t r = 1;
    while (e) {
      if (e & 1) r = mulmod(r, a);
      a = mulmod(a, a);
      e >>= 1;
    }
    return r;
  };
  for (uint64_t a : {2ull, 3ull, 5ull, 7ull, 11ull, 13ull, 17ull, 19ull, 23ull, 29ull, 31ull, 37ull}) {
    uint64_t x = powmod(a, d);
    if (x == 1 || x == n - 1) continue;
    bool comp = true;
    for (int r = 1; r < s; ++r) {
      x = mulmod(x, x);
      if (x == n - 1) {
        comp = false;
        break;
      }
    }
    if (comp) return false;
  }
  return true;
}
bool prime_check(uint64_t n) { return is_prime_u64(n); }

static int validate_poly(const qmc_poly& p, int d, const char* name) {
  if (p.nterms < 1 || p.nterms > kTermsMax)
    return fail(QMC_EINVAL, "%s: nterms=%d outside [1, %d]", name, p.nterms, kTermsMax);
  if (!p.coef || !p.expo) return fail(QMC_EINVAL, "%s: null coefficient or exponent table", name);
  for (int t = 0; t < p.nterms; ++t) {
    if (!std::isfinite(p.coef[t])) return fail(QMC_EINVAL, "%s: coefficient %d not finite", name, t);
    int deg = 0;
    for (int i = 0; i < d; ++i) deg += p.expo[(size_t)t * d + i];
    if (deg > 3) return fail(QMC_EINVAL, "%s: term %d has degree %d > 3", name, t, deg);
  }
  return QMC_OK;
}

int validate_problem(int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts,
                     const qmc_transform& t, const qmc_integrand* f) {
  if (d < 1 || d > QMC_DMAX) return fail(QMC_EINVAL, "d=%d outside [1, %d]", d, QMC_DMAX);
  if (n < 2 || n >= (1ull << 31)) return fail(QMC_EINVAL, "n=%llu outside [2, 2^31)", (unsigned long long)n);
  if (m < 2 || m > 1024) return fail(QMC_EINVAL, "m=%d outside [2, 1024] (Eq. 3 needs m >= 2)", m);
  if (!g || !shifts || !f) return fail(QMC_EINVAL, "null g, shifts or integrand");
  for (int i = 0; i < d; ++i)
    if (g[i] < 1 || g[i] >= n) return fail(QMC_EINVAL, "g[%d]=%llu outside [1, n)", i, (unsigned long long)g[i]);
  for (int k = 0; k < m * d; ++k)
    if (!(shifts[k] >= 0.0 && shifts[k] < 1.0)) return fail(QMC_EINVAL, "shift entry %d outside [0, 1)", k);
  if (t.kind != QMC_TRANSFORM_NONE && t.kind != QMC_TRANSFORM_KOROBOV && t.kind != QMC_TRANSFORM_BAKER)
    return fail(QMC_EINVAL, "unknown transform %d", t.kind);
  if (t.kind == QMC_TRANSFORM_KOROBOV && (t.alpha < 1 || t.alpha > 6))
    return fail(QMC_EINVAL, "Korobov weight %d outside [1, 6]", t.alpha);
  if (f->d != d) return fail(QMC_EINVAL, "integrand d=%d differs from rule d=%d", f->d, d);
  if (f->precision != QMC_FP64 && f->precision != QMC_FP32EVAL)
    return fail(QMC_EINVAL, "unknown precision %d", f->precision);
  switch (f->kind) {
    case QMC_F_CONST:
      break;
    case QMC_F_SEPARABLE_EXP:
      if (!f->c || !f->b) return fail(QMC_EINVAL, "separable integrand needs c and b");
      for (int i = 0; i < d; ++i)
        if (!std::isfinite(f->c[i]) || !std::isfinite(f->b[i]))
          return fail(QMC_EINVAL, "separable coefficient %d not finite", i);
      break;
    case QMC_F_TRIG:
      if (!f->h) return fail(QMC_EINVAL, "trig integrand needs h");
      break;
    case QMC_F_SECTOR:
    case QMC_F_SECTOR_DEFORMED: {
      int rc = validate_poly(f->U, d, "U");
      if (rc) return rc;
      rc = validate_poly(f->F, d, "F");
      if (rc) return rc;
      if (f->aU < -8 || f->aU > 8 || f->aF < -8 || f->aF > 8)
        return fail(QMC_EINVAL, "powers aU=%d aF=%d outside [-8, 8]", f->aU, f->aF);
      if (f->kind == QMC_F_SECTOR_DEFORMED) {
        if (!std::isfinite(f->lambda) || f->lambda < 0.0)
          return fail(QMC_EINVAL, "deformation lambda must be finite and >= 0");
        for (int t2 = 0; t2 < f->F.nterms; ++t2) {
          int deg = 0;
          for (int i = 0; i < d; ++i) deg += f->F.expo[(size_t)t2 * d + i];
          if (deg > 2) return fail(QMC_EINVAL, "deformed F must have degree <= 2");
        }
        for (int t2 = 0; t2 < f->U.nterms; ++t2) {
          int deg = 0;
          for (int i = 0; i < d; ++i) deg += f->U.expo[(size_t)t2 * d + i];
          if (deg > 2) return fail(QMC_EINVAL, "deformed U must have degree <= 2");
        }
      }
      break;
    }
    default:
      return fail(QMC_EINVAL, "unknown integrand kind %d", f->kind);
  }
  return QMC_OK;
}

// ---------------------------------------------------------------- packing --

int poly_degree(const qmc_poly& p, int d) {
  int deg = 0;
  for (int t = 0; t < p.nterms; ++t) {
    int s = 0;
    for (int i = 0; i < d; ++i) s += p.expo[(size_t)t * d + i];
    deg = std::max(deg, s);
  }
  return deg;
}

// Coefficient of every monomial (sorted variable list, repeated monomials summed).
static std::map<std::vector<int>, double> monomials(const qmc_poly& p, int d) {
  std::map<std::vector<int>, double> out;
  for (int t = 0; t < p.nterms; ++t) {
    std::vector<int> vars;
    for (int i = 0; i < d; ++i)
      for (int e = 0; e < p.expo[(size_t)t * d + i]; ++e) vars.push_back(i);
    out[vars] += p.coef[t];
  }
  return out;
}

// Nested-Horner slots of a degree-K polynomial in D variables (order matches
// poly_dense): c0; for i: l_i, [K>=2: for j>=i: q_ij, [K=3: c_ijk for k>=j]].
std::vector<double> pack_dense(const qmc_poly& p, int D, int K) {
  auto mono = monomials(p, D);
  auto get = [&](std::vector<int> v) {
    auto it = mono.find(v);
    return it == mono.end() ? 0.0 : it->second;
  };
  std::vector<double> c;
  c.push_back(get({}));
  if (K == 1) {
    for (int i = 0; i < D; ++i) c.push_back(get({i}));
  } else if (K == 2) {
    for (int i = 0; i < D; ++i) {
      c.push_back(get({i}));
      for (int j = i; j < D; ++j) c.push_back(get({i, j}));
    }
  } else if (K == 3) {
    for (int i = 0; i < D; ++i) {
      c.push_back(get({i}));
      for (int j = i; j < D; ++j) {
        c.push_back(get({i, j}));
        for (int k = j; k < D; ++k) c.push_back(get({i, j, k}));
      }
    }
  }
  return c;
}

// 2^128 / n = rhi 2^64 + rlo + frac
Recip reciprocal(uint64_t n) {
  unsigned __int128 one64 = (unsigned __int128)1 << 64;
  Recip r;
  r.rhi = (uint64_t)(one64 / n);
  uint64_t rem = (uint64_t)(one64 % n);
  r.rlo = (uint64_t)(((unsigned __int128)rem << 64) / n);
  return r;
}

// Korobov z(s) = C sum_k binom(a,k) (-1)^k s^(a+k+1)/(a+k+1), C = (2a+1)!/(a!)^2.
void korobov_coefs(int alpha, double* kor /*8*/) {
  double C = 1.0;
  for (int i = 1; i <= 2 * alpha + 1; ++i) C *= (double)i;
  double f = 1.0;
  for (int i = 1; i <= alpha; ++i) f *= (double)i;
  C /= f * f;
  for (int k = 0; k < 8; ++k) kor[k] = 0.0;
  for (int k = 0; k <= alpha; ++k) {
    double b = 1.0;
    for (int i = 1; i <= k; ++i) b = b * (double)(alpha - k + i) / (double)i;
    kor[k] = ((k & 1) ? -1.0 : 1.0) * C * b / (double)(alpha + k + 1);
  }
  kor[7] = C;
}

uint64_t shift_fixed64(double delta) {
  // delta in [0, 1): delta * 2^64, floor
  long double v = std::ldexp((long double)delta, 64);
  if (v >= 18446744073709551615.0L) return ~0ull;
  return (uint64_t)v;
}

// Positive on the cube: a positive constant term and no negative coefficient.
bool poly_positive(const qmc_poly& p, int d) {
  bool has_const = false;
  for (int t = 0; t < p.nterms; ++t) {
    int deg = 0;
    for (int i = 0; i < d; ++i) deg += p.expo[(size_t)t * d + i];
    if (p.coef[t] < 0.0) return false;
    if (deg == 0 && p.coef[t] > 0.0) has_const = true;
  }
  return has_const;
}

template <typename R>
void fill_common(RuleParams<R>& P, int32_t d, uint64_t n, const uint64_t* g, const qmc_transform& t,
                 const qmc_integrand* f) {
  std::memset(&P, 0, sizeof(P));
  P.n = n;
  P.d = d;
  P.alpha = t.kind == QMC_TRANSFORM_KOROBOV ? t.alpha : 0;
  P.tr = t.kind == QMC_TRANSFORM_KOROBOV ? TR_KOROBOV : (t.kind == QMC_TRANSFORM_BAKER ? TR_BAKER : TR_NONE);
  P.aU = f->aU;
  P.aF = f->aF;
  P.lam = (R)f->lambda;
  P.value_scale = 1.0;
  P.rc = reciprocal(n);
  for (int i = 0; i < d; ++i) {
    P.g[i] = (uint32_t)g[i];
    P.gstep[i] = (uint32_t)(((uint64_t)kThreads * g[i]) % n);
  }
  double kor[8];
  korobov_coefs(P.alpha > 0 ? P.alpha : 1, kor);
  for (int k = 0; k < 8; ++k) P.kor[k] = (R)kor[k];
  if (f->kind == QMC_F_SEPARABLE_EXP) {
    for (int i = 0; i < d; ++i) {
      P.sep_c[i] = (R)f->c[i];
      P.sep_b[i] = (R)f->b[i];
    }
  } else if (f->kind == QMC_F_TRIG) {
    for (int i = 0; i < d; ++i) P.sep_c[i] = (R)f->h[i];
  }
  P.check_finite = 1;
  if (f->kind == QMC_F_CONST) P.check_finite = 0;
  if (f->kind == QMC_F_SECTOR && f->aU <= 0 && f->aF <= 0 && poly_positive(f->U, d) && poly_positive(f->F, d))
    P.check_finite = 0;
}

// ------------------------------------------------------------------- plan --

// SM count of the current device, read once per device (plans query it for
// every launch shape, a walk for every sector and pass).
static int device_sm_count() {
  constexpr int kMaxDevices = 64;
  static std::atomic<int> cache[kMaxDevices];
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -1;
  if (dev >= 0 && dev < kMaxDevices && (sms = cache[dev].load(std::memory_order_relaxed)) > 0) return sms;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -1;
  if (dev >= 0 && dev < kMaxDevices) cache[dev].store(sms, std::memory_order_relaxed);
  return sms;
}

int device_sms() { return device_sm_count(); }

// CTAs of `func` resident per SM (at least 1), capped by occupancy_override
// when > 0; a run-time compiled kernel (func null) takes the caller's figure.
int grid_occupancy(const void* func, size_t smem, int occupancy_override, int& occ) {
  occ = 0;
  if (func) {
    QMC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, func, kThreads, smem));
    if (occ < 1) occ = 1;
    if (occupancy_override > 0) occ = std::min(occ, occupancy_override);
  } else {
    occ = std::max(1, occupancy_override);
  }
  return QMC_OK;
}

// Grid: one resident wave (SMs x occ CTAs), each CTA one tile of kThreads * L
// points, L from the point count; then at most max_ctas CTAs (> 0) and a
// fixed L (> 0) if asked.
int grid_shape(int occ, uint64_t n, int max_ctas, int fixed_L, int& nblk, int& L, uint64_t& tiles) {
  const int sms = device_sm_count();
  if (sms <= 0) return fail(QMC_ECUDA, "no CUDA device");
  const uint64_t Lmax = 512;
  const uint64_t want = (uint64_t)sms * (uint64_t)std::max(occ, 1);
  uint64_t per = (n + want * kThreads - 1) / (want * kThreads);
  L = (int)std::max<uint64_t>(1, std::min(per, Lmax));
  tiles = (n + (uint64_t)kThreads * L - 1) / ((uint64_t)kThreads * L);
  nblk = (int)std::min<uint64_t>(want, tiles);
  if (max_ctas > 0 && nblk > max_ctas) {
    nblk = max_ctas;
    per = (n + (uint64_t)nblk * kThreads - 1) / ((uint64_t)nblk * kThreads);
    L = (int)std::max<uint64_t>(1, std::min(per, Lmax));
    tiles = (n + (uint64_t)kThreads * L - 1) / ((uint64_t)kThreads * L);
    nblk = (int)std::min<uint64_t>((uint64_t)nblk, tiles);
  }
  if (fixed_L > 0) {
    L = fixed_L;
    tiles = (n + (uint64_t)kThreads * L - 1) / ((uint64_t)kThreads * L);
    nblk = (int)std::min<uint64_t>((uint64_t)nblk, tiles);
  }
  return QMC_OK;
}

int choose_grid(const void* func, size_t smem, uint64_t n, int& nblk, int& L, uint64_t& tiles,
                int occupancy_override) {
  int occ = 0;
  int rc = grid_occupancy(func, smem, occupancy_override, occ);
  if (rc) return rc;
  return grid_shape(occ, n, 0, 0, nblk, L, tiles);
}

static int pick_mc(int m, bool fp32) {
  if (!fp32) return 16;
  int mm = std::min(m, kMcMax);
  if (mm <= 8) return 8;
  if (mm <= 16) return 16;
  return 32;
}

template <typename R>
static int build_rule_plan(Plan* pl, int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts,
                           const qmc_transform& t, const qmc_integrand* f, const TuneChoice& tune,
                           const qmc_eps* eps) {
  const bool fp32 = sizeof(R) == 4;
  RuleParams<R> base;
  fill_common(base, d, n, g, t, f);
  const void* func = nullptr;
  void* jit_fn = nullptr;
  int jit_occ = 0;
  size_t jit_smem = 0;
  size_t pbytes = sizeof(RuleParams<R>);
  std::vector<uint8_t> blob;
  int mc = tune.mc > 0 ? tune.mc : pick_mc(m, fp32);
  bool general = false;

  if (eps) {
    // Eq. (7) expansion: 3 or kEpsMax orders per pass, kEpsAcc sums per thread
    base.eps_orders = eps->orders;
    base.m_total = m;
    base.eps_b[0] = (R)eps->bU;
    base.eps_b[1] = (R)eps->bF;
    for (int k = 0; k < kEpsMax; ++k) base.eps_inv[k] = (R)(1.0 / (double)(k + 1));
    const int ne = eps->orders <= 3 ? 3 : kEpsMax;
    const int ku = poly_degree(f->U, d), kf = poly_degree(f->F, d);
    const bool fast_tr = base.tr == TR_BAKER || (base.tr == TR_KOROBOV && base.alpha == 3);
    if (ku <= 1 && kf <= 2 && f->aU == -2 && f->aF == -1 && d <= kDFast && fast_tr && !tune.force_general) {
      switch (d) {
#define QMC_D_CASE(DD) \
  case DD:             \
    func = eps_ptr<R, DD>(ne, base.tr); \
    break;
        QMC_D_CASE(1) QMC_D_CASE(2) QMC_D_CASE(3) QMC_D_CASE(4) QMC_D_CASE(5) QMC_D_CASE(6)
        QMC_D_CASE(7) QMC_D_CASE(8)
#undef QMC_D_CASE
        default: break;
      }
    }
    if (func) {
      mc = kEpsAcc / ne;
      auto cu = pack_dense(f->U, d, 1);
      auto cf = pack_dense(f->F, d, 2);
      if (fp32) {
        prescale_slots(cu.data(), d, 1, fx_sigma(base.tr));
        prescale_slots(cf.data(), d, 2, fx_sigma(base.tr));
      }
      for (size_t i = 0; i < cu.size(); ++i) base.cU[i] = (R)cu[i];
      for (size_t i = 0; i < cf.size(); ++i) base.cF[i] = (R)cf[i];
      if (base.tr == TR_KOROBOV) base.value_scale = std::pow((double)base.kor[7], (double)d);
      if (fp32 && !tune.no_jit && jit_enabled()) {
        // run-time specialised, packed, exactly `orders` orders; one logarithm
        // per value when U, F > 0 on the cube and bF = -bU
        fill_pairs(base, d);
        const int NE = eps->orders;
        const int jmc = NE <= 2 ? 16 : (NE <= 3 ? 8 : 4);
        const bool positive = base.check_finite == 0;
        const bool log1 = positive && eps->bF == -eps->bU;
        void* fn = nullptr;
        int occ = 0;
        if (jit_eps_f32(d, jmc, NE, base.tr, base.tr == TR_KOROBOV ? 3 : 0, log1, !positive, cu, cf, &fn, &occ) ==
            QMC_OK) {
          jit_fn = fn;
          jit_occ = occ;
          mc = jmc;
        }
      }
    } else {
      general = true;
    }
  } else if (f->kind == QMC_F_SECTOR) {
    int ku = poly_degree(f->U, d), kf = poly_degree(f->F, d);
    int KU = -1, KF = -1;
    if (ku <= 1 && kf <= 2) {
      KU = 1;
      KF = 2;
    } else if (ku <= 2 && kf <= 3 && fp32) {
      KU = 2;
      KF = 3;
      mc = 16;
    }
    const bool m21 = f->aU == -2 && f->aF == -1;
    if (KU > 0 && d <= kDFast && m21 && !tune.force_general) {
      switch (d) {
#define QMC_D_CASE(DD) \
  case DD:             \
    func = sector_ptr<R, DD>(mc, base.tr, base.alpha, KU, KF, base.check_finite != 0); \
    break;
        QMC_D_CASE(1) QMC_D_CASE(2) QMC_D_CASE(3) QMC_D_CASE(4) QMC_D_CASE(5) QMC_D_CASE(6)
        QMC_D_CASE(7) QMC_D_CASE(8)
#undef QMC_D_CASE
        default: break;
      }
    }
    if (func) {
      auto cu = pack_dense(f->U, d, KU);
      auto cf = pack_dense(f->F, d, KF);
      if (fp32) {  // the FP32 kernels hand the polynomials z / fx_sigma (exact powers of two)
        prescale_slots(cu.data(), d, KU, fx_sigma(base.tr));
        prescale_slots(cf.data(), d, KF, fx_sigma(base.tr));
      }
      for (size_t i = 0; i < cu.size(); ++i) base.cU[i] = (R)cu[i];
      for (size_t i = 0; i < cf.size(); ++i) base.cF[i] = (R)cf[i];
      if (fp32 && KU == 1 && KF == 2) fill_pairs(base, d);
      if (base.tr == TR_KOROBOV) base.value_scale = std::pow((double)base.kor[7], (double)d);
      if (fp32 && KU == 1 && KF == 2 && !tune.no_jit && jit_enabled()) {
        void* fn = nullptr;
        int occ = 0;
        size_t sm = 0;
        const bool smacc = tune.smacc < 0 ? jit_smacc() : tune.smacc != 0;
        // shifts as immediate operands: one compiled kernel per shift table, so
        // only for plans of one launch chunk, and only when the tuner asks
        std::vector<uint32_t> imm;
        bool use_imm = tune.imm < 0 ? jit_imm() : tune.imm != 0;
        if (use_imm && m > mc) {
          if (tune.imm == 1) return fail(QMC_EUNSUPPORTED, "immediate shifts need one launch chunk (m <= %d)", mc);
          use_imm = false;
        }
        if (use_imm) {
          imm.resize((size_t)mc * d);
          for (int kk = 0; kk < mc; ++kk)
            for (int i = 0; i < d; ++i)
              imm[(size_t)kk * d + i] =
                  (uint32_t)((shift_fixed64(shifts[(size_t)(kk < m ? kk : 0) * d + i]) + 0x80000000ull) >> 32);
        }
        if (jit_sector_f32(d, mc, base.tr, base.tr == TR_KOROBOV ? 3 : 0, base.check_finite != 0, cu, cf, smacc,
                           tune.minb, &fn, &occ, &sm, use_imm ? imm.data() : nullptr) == QMC_OK) {
          pl->imm = use_imm ? 1 : 0;
          jit_fn = fn;
          jit_occ = occ;
          jit_smem = sm;
        }
      }
    } else {
      general = true;
    }
  } else if (f->kind == QMC_F_SECTOR_DEFORMED) {
    return fail(QMC_EUNSUPPORTED, "deformed sector integrands are served by the complex kernels");
  } else {
    int fk = f->kind == QMC_F_CONST ? FK_CONST : (f->kind == QMC_F_SEPARABLE_EXP ? FK_SEPEXP : FK_TRIG);
    mc = 8;
    func = separable_ptr(fp32, base.tr, fk);
    if (!func) return fail(QMC_EUNSUPPORTED, "no separable kernel for this transform");
  }

  GeneralParams<R> gp;
  if (general) {
    mc = eps ? kEpsAcc / kEpsMax : 8;
    std::memset(&gp, 0, sizeof(gp));
    func = eps ? general_eps_ptr(fp32) : general_ptr(fp32);
    pbytes = sizeof(GeneralParams<R>);
    auto fill_sparse = [&](SparsePoly<R>& S, const qmc_poly& p) {
      S.nterms = p.nterms;
      for (int tt = 0; tt < p.nterms; ++tt) {
        S.coef[tt] = (R)p.coef[tt];
        for (int i = 0; i < d; ++i) S.expo[tt][i] = p.expo[(size_t)tt * d + i];
      }
    };
    fill_sparse(gp.U, f->U);
    fill_sparse(gp.F, f->F);
  }
  // FP32 float-coordinate kernels (general, separable) raise the product of the
  // Korobov factors 4u to the power alpha once per value: the constant
  // ((2a+1)!/(a!)^2 / 4^a) per dimension is applied in FP64 by the final pass
  if (fp32 && (general || !(f->kind == QMC_F_SECTOR || eps)) && base.tr == TR_KOROBOV)
    base.value_scale = std::pow((double)base.kor[7] / std::pow(4.0, (double)base.alpha), (double)d);

  int nblk = 0, L = 0, occ = 0;
  uint64_t tiles = 0;
  // a run-time specialised kernel has its own occupancy (registers, shared memory), not the template's
  int rc = grid_occupancy(jit_fn ? nullptr : func, 0,
                          jit_fn ? (tune.occupancy > 0 ? std::min(tune.occupancy, jit_occ) : jit_occ)
                                 : tune.occupancy,
                          occ);
  if (rc) return rc;
  rc = grid_shape(occ, n, tune.max_ctas, tune.L, nblk, L, tiles);
  if (rc) return rc;
  pl->param_kind = general ? (fp32 ? 3 : 4) : (fp32 ? 1 : 2);
  pl->grid_occ = occ;
  pl->grid_capped = true;
  base.L = L;
  base.tiles = tiles;
  base.nblk = nblk;
  pl->nblk = nblk;
  pl->func = func;
  pl->mc = mc;
  pl->value_scale = 1.0;  // applied per value inside the kernels' sums via finalize
  pl->final_scale = base.value_scale;
  for (int k0 = 0; k0 < m; k0 += mc) {
    int mk = std::min(mc, m - k0);
    RuleParams<R> P = base;
    P.m_launch = mk;
    P.k_base = k0;
    // rows mk..mc-1 repeat row 0 (evaluated, never written back)
    for (int kk = 0; kk < mc; ++kk)
      for (int i = 0; i < d; ++i) {
        const int src = kk < mk ? k0 + kk : k0;
        uint64_t s64 = shift_fixed64(shifts[(size_t)src * d + i]);
        set_shift(P, kk, i, s64);
      }
    Launch ln;
    ln.func = func;
    ln.cufunc = jit_fn;
    ln.smem = jit_fn ? jit_smem : 0;
    ln.grid = dim3(nblk);
    ln.params.resize(pbytes);
    if (general) {
      gp.base = P;
      std::memcpy(ln.params.data(), &gp, pbytes);
    } else {
      std::memcpy(ln.params.data(), &P, pbytes);
    }
    pl->launches.push_back(std::move(ln));
  }
  return QMC_OK;
}

void SavedProblem::save(int32_t d_, uint64_t n_, int32_t m_, const uint64_t* g_, const double* shifts_,
                        qmc_transform t_, const qmc_integrand* f_) {
  d = d_;
  n = n_;
  m = m_;
  t = t_;
  g.assign(g_, g_ + d_);
  shifts.assign(shifts_, shifts_ + (size_t)m_ * d_);
  f = *f_;
  auto copy_poly = [&](qmc_poly& p, std::vector<double>& cv, std::vector<uint8_t>& ev) {
    if (p.nterms > 0 && p.coef && p.expo) {
      cv.assign(p.coef, p.coef + p.nterms);
      ev.assign(p.expo, p.expo + (size_t)p.nterms * d_);
      p.coef = cv.data();
      p.expo = ev.data();
    }
  };
  copy_poly(f.U, cu, eu);
  copy_poly(f.F, cf, ef);
  if (f_->c) {
    c.assign(f_->c, f_->c + d_);
    f.c = c.data();
  }
  if (f_->b) {
    b.assign(f_->b, f_->b + d_);
    f.b = b.data();
  }
  if (f_->h) {
    h.assign(f_->h, f_->h + d_);
    f.h = h.data();
  }
}

int plan_build(Plan* pl, int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts,
               qmc_transform t, const qmc_integrand* f, const TuneChoice& tune, const qmc_eps* eps) {
  int rc = validate_problem(d, n, m, g, shifts, t, f);
  if (rc) return rc;
  if (eps) {
    if (eps->orders < 1 || eps->orders > kEpsMax)
      return fail(QMC_EINVAL, "epsilon orders %d outside [1, %d]", eps->orders, kEpsMax);
    if (!std::isfinite(eps->bU) || !std::isfinite(eps->bF)) return fail(QMC_EINVAL, "non-finite epsilon slopes");
    if (f->kind != QMC_F_SECTOR) return fail(QMC_EINVAL, "the epsilon expansion applies to SECTOR integrands");
  }
  pl->orders = eps ? eps->orders : 1;
  pl->tune = tune;
  pl->d = d;
  pl->n = n;
  pl->m = m;
  pl->is_complex = f->kind == QMC_F_SECTOR_DEFORMED;
  if (f->kind == QMC_F_SECTOR_DEFORMED) {
    rc = build_deformed_plan(pl, d, n, m, g, shifts, t, f, tune);
  } else if (f->precision == QMC_FP32EVAL) {
    rc = build_rule_plan<float>(pl, d, n, m, g, shifts, t, f, tune, eps);
  } else {
    rc = build_rule_plan<double>(pl, d, n, m, g, shifts, t, f, tune, eps);
  }
  return rc;
}

template <typename R>
static void rebase_rule(RuleParams<R>& P, int d, uint64_t n, const uint64_t* g, int nblk, int L, uint64_t tiles) {
  P.n = n;
  P.rc = reciprocal(n);
  for (int i = 0; i < d; ++i) {
    P.g[i] = (uint32_t)g[i];
    P.gstep[i] = (uint32_t)(((uint64_t)kThreads * g[i]) % n);
  }
  P.L = L;
  P.tiles = tiles;
  P.nblk = nblk;
}

int plan_rebase(Plan* pl, uint64_t n, const uint64_t* g, int max_ctas) {
  if (pl->param_kind < 1 || pl->param_kind > 4) return fail(QMC_EUNSUPPORTED, "this plan is bound to its lattice");
  if (n < 2 || n >= (1ull << 31)) return fail(QMC_EINVAL, "n=%llu outside [2, 2^31)", (unsigned long long)n);
  for (int i = 0; i < pl->d; ++i)
    if (g[i] < 1 || g[i] >= n) return fail(QMC_EINVAL, "g[%d]=%llu outside [1, n)", i, (unsigned long long)g[i]);
  int nblk = 0, L = 0;
  uint64_t tiles = 0;
  int rc = grid_shape(pl->grid_occ, n, pl->grid_capped ? max_ctas : 0, pl->tune.L, nblk, L, tiles);
  if (rc) return rc;
  for (Launch& ln : pl->launches) {
    uint8_t* p = ln.params.data();
    switch (pl->param_kind) {
      case 1: rebase_rule(*reinterpret_cast<RuleParams<float>*>(p), pl->d, n, g, nblk, L, tiles); break;
      case 2: rebase_rule(*reinterpret_cast<RuleParams<double>*>(p), pl->d, n, g, nblk, L, tiles); break;
      case 3: rebase_rule(reinterpret_cast<GeneralParams<float>*>(p)->base, pl->d, n, g, nblk, L, tiles); break;
      default: rebase_rule(reinterpret_cast<GeneralParams<double>*>(p)->base, pl->d, n, g, nblk, L, tiles); break;
    }
    ln.grid = dim3(nblk);
  }
  pl->n = n;
  pl->nblk = nblk;
  pl->tune.max_ctas = max_ctas;
  return QMC_OK;
}

template <typename R>
static void reshift_rule(RuleParams<R>& P, int d, int mc, const double* shifts) {
  // rows m_launch..mc-1 repeat the launch's first row, as at build time
  for (int kk = 0; kk < mc; ++kk)
    for (int i = 0; i < d; ++i) {
      const int src = kk < P.m_launch ? P.k_base + kk : P.k_base;
      set_shift(P, kk, i, shift_fixed64(shifts[(size_t)src * d + i]));
    }
}

int plan_reshift(Plan* pl, const double* shifts) {
  if (pl->param_kind < 1 || pl->param_kind > 4) return fail(QMC_EUNSUPPORTED, "this plan is bound to its shifts");
  if (pl->imm) return fail(QMC_EUNSUPPORTED, "this plan has its shifts compiled into its kernel");
  for (size_t u = 0; u < (size_t)pl->m * pl->d; ++u)
    if (!(shifts[u] >= 0.0 && shifts[u] < 1.0)) return fail(QMC_EINVAL, "shift value %zu outside [0, 1)", u);
  for (Launch& ln : pl->launches) {
    uint8_t* p = ln.params.data();
    switch (pl->param_kind) {
      case 1: reshift_rule(*reinterpret_cast<RuleParams<float>*>(p), pl->d, pl->mc, shifts); break;
      case 2: reshift_rule(*reinterpret_cast<RuleParams<double>*>(p), pl->d, pl->mc, shifts); break;
      case 3: reshift_rule(reinterpret_cast<GeneralParams<float>*>(p)->base, pl->d, pl->mc, shifts); break;
      default: reshift_rule(reinterpret_cast<GeneralParams<double>*>(p)->base, pl->d, pl->mc, shifts); break;
    }
  }
  return QMC_OK;
}

int plan_alloc(Plan* pl, cudaStream_t stream, bool async) {
  const size_t G = (size_t)pl->orders;
  size_t partial_bytes = G * pl->m * pl->nblk * 2 * sizeof(double);
  size_t total = partial_bytes + G * (2 * sizeof(unsigned long long) + sizeof(qmc_result) + (size_t)pl->m * 2 * sizeof(double)) + 256;
  void* p = nullptr;
  cudaError_t e = async ? cudaMallocAsync(&p, total, stream) : cudaMalloc(&p, total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(QMC_ENOMEM, "device workspace of %zu bytes: %s", total, cudaGetErrorString(e));
  }
  pl->ws_base = p;
  pl->ws_async = async;
  char* c = (char*)p;
  pl->ws.partial = (double*)c;
  c += partial_bytes;
  pl->ws.counters = (unsigned long long*)c;
  c += G * 2 * sizeof(unsigned long long);
  pl->ws.result = (qmc_result*)c;
  c += G * sizeof(qmc_result);
  c = (char*)(((uintptr_t)c + 15) & ~(uintptr_t)15);
  pl->ws.per_shift = (double*)c;
  e = async ? cudaMemsetAsync(pl->ws.counters, 0, G * 2 * sizeof(unsigned long long), stream)
            : cudaMemset(pl->ws.counters, 0, G * 2 * sizeof(unsigned long long));
  if (e != cudaSuccess) return cuda_fail(e, "clear counters");
  return QMC_OK;
}

void plan_free(Plan* pl, cudaStream_t stream) {
  if (!pl->ws_base) return;
  if (pl->ws_async) cudaFreeAsync(pl->ws_base, stream);
  else cudaFree(pl->ws_base);
  pl->ws_base = nullptr;
}

int launch_rule(const Plan* pl, const Workspace& ws, cudaStream_t stream, const SampleIO& sio) {
  for (const Launch& ln : pl->launches) {
    void* args[4];
    args[0] = (void*)ln.params.data();
    double* partial = ws.partial;
    unsigned long long* counters = ws.counters;
    args[1] = &partial;
    args[2] = &counters;
    args[3] = (void*)&sio;
    int rc = launch_any(ln, ln.grid, args, stream);
    if (rc) return rc;
  }
  return QMC_OK;
}

int launch_finalize(const Plan* pl, const Workspace& ws, qmc_result* res_dev, double* per_shift_dev,
                    cudaStream_t stream) {
  FinalizeArgs A;
  A.partial = ws.partial;
  A.nblk = pl->nblk;
  A.m = pl->m;
  A.is_complex = pl->is_complex;
  A.groups = pl->orders;
  A.sum_last = pl->sum_last ? 1 : 0;
  A.pad = 0;
  A.dn = (double)pl->n;
  A.value_scale = pl->final_scale;
  A.offset[0] = pl->offset[0];
  A.offset[1] = pl->offset[1];
  A.counters = ws.counters;
  A.result = res_dev;
  A.per_shift = per_shift_dev;
  void* args[1] = {&A};
  size_t smem = (size_t)pl->m * 2 * sizeof(double);
  QMC_CUDA(cudaLaunchKernel(finalize_ptr(), dim3(pl->orders), dim3(256), args, smem, stream));
  return QMC_OK;
}

int plan_execute(Plan* pl, qmc_result* out, double* per_shift, cudaStream_t stream) {
  if (!out) return fail(QMC_EINVAL, "null result pointer");
  const bool out_dev = is_device_pointer(out);
  const bool ps_dev = per_shift ? is_device_pointer(per_shift) : true;
  SampleIO none;
  std::memset(&none, 0, sizeof(none));
  if (pl->ev_before) QMC_CUDA(cudaEventRecord(pl->ev_before, stream));
  int rc = launch_rule(pl, pl->ws, stream, none);
  if (rc) return rc;
  if (pl->ev_after) QMC_CUDA(cudaEventRecord(pl->ev_after, stream));
  rc = launch_finalize(pl, pl->ws, out_dev ? out : pl->ws.result,
                       (per_shift && ps_dev) ? per_shift : (per_shift ? pl->ws.per_shift : nullptr), stream);
  if (rc) return rc;
  const size_t G = (size_t)pl->orders;
  if (!out_dev) QMC_CUDA(cudaMemcpyAsync(out, pl->ws.result, G * sizeof(qmc_result), cudaMemcpyDeviceToHost, stream));
  if (per_shift && !ps_dev)
    QMC_CUDA(cudaMemcpyAsync(per_shift, pl->ws.per_shift, G * pl->m * 2 * sizeof(double),
                             cudaMemcpyDeviceToHost, stream));
  if (!out_dev || (per_shift && !ps_dev)) {
    QMC_CUDA(cudaStreamSynchronize(stream));
    if (!out_dev) {
      // the first failing order's status (NaN/Inf values are counted per order)
      for (size_t o = 0; o < G; ++o)
        if (out[o].status != QMC_OK) return out[o].status;
      return QMC_OK;
    }
  }
  return QMC_OK;
}

}  // namespace qmc

using namespace qmc;

// ------------------------------------------------------------------ C ABI --

extern "C" {

const char* qmc_last_error(void) { return g_last_error.c_str(); }

int32_t qmc_version(void) { return 100; }

int qmc_plan_create(int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts, qmc_transform t,
                    const qmc_integrand* f, qmc_plan* plan_out) {
  if (!plan_out) return fail(QMC_EINVAL, "null plan_out");
  *plan_out = nullptr;
  std::unique_ptr<Plan> pl(new Plan());
  int rc = plan_build(pl.get(), d, n, m, g, shifts, t, f, TuneChoice{});
  if (rc) return rc;
  rc = plan_alloc(pl.get(), nullptr, false);
  if (rc) return rc;
  pl->saved.save(d, n, m, g, shifts, t, f);
  *plan_out = reinterpret_cast<qmc_plan>(pl.release());
  return QMC_OK;
}

int qmc_plan_tune(qmc_plan plan, void* stream, int32_t* shifts_per_launch_out) {
  if (!plan) return fail(QMC_EINVAL, "null plan");
  Plan* pl = reinterpret_cast<Plan*>(plan);
  cudaStream_t st = (cudaStream_t)stream;
  const SavedProblem& sp = pl->saved;
  // candidates (shifts per launch, accumulators in shared memory, min CTAs per SM)
  struct Cand {
    int mc, smacc, minb, imm;
  };
  std::vector<Cand> cands;
  if (sp.f.precision == QMC_FP32EVAL && sp.f.kind == QMC_F_SECTOR && sp.eps.orders == 0) {
    cands = {{8, 0, 0, 0}, {16, 0, 0, 0}, {32, 0, 0, 0}};
    if (pl->launches.size() && pl->launches[0].cufunc) {
      // register-pressure variants of the specialised kernel
      cands.insert(cands.end(), {{16, 0, 2, 0}, {16, 1, 2, 0}, {32, 1, 0, 0}, {32, 1, 2, 0}, {32, 0, 2, 0}});
    }
  }
  if (cands.empty()) {
    if (shifts_per_launch_out) *shifts_per_launch_out = pl->mc;
    return QMC_OK;
  }
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return fail(QMC_ECUDA, "events");
  qmc_result* dres = nullptr;
  QMC_CUDA(cudaMalloc(&dres, sizeof(qmc_result)));
  float best = 1e30f;
  Cand best_c{pl->mc, pl->tune.smacc, pl->tune.minb, pl->imm};
  int rc = QMC_OK;
  const char* ve = std::getenv("QMC_TUNE_VERBOSE");  // per-candidate times on stderr
  const bool verbose = ve && ve[0] == '1';
  for (const Cand& cd : cands) {
    Plan trial;
    TuneChoice tc = pl->tune;
    tc.mc = cd.mc;
    tc.smacc = cd.smacc;
    tc.minb = cd.minb;
    tc.imm = cd.imm;
    rc = plan_build(&trial, sp.d, sp.n, sp.m, sp.g.data(), sp.shifts.data(), sp.t, &sp.f, tc);
    if (rc == QMC_EUNSUPPORTED) {
      rc = QMC_OK;
      continue;
    }
    if (rc) break;
    rc = plan_alloc(&trial, nullptr, false);
    if (rc) break;
    float tot = 0.0f;
    for (int rep = 0; rep < 4 && rc == QMC_OK; ++rep) {
      cudaEventRecord(a, st);
      rc = plan_execute(&trial, dres, nullptr, st);
      cudaEventRecord(b, st);
      cudaEventSynchronize(b);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, a, b);
      if (rep > 0) tot += ms;
    }
    plan_free(&trial, nullptr);
    if (rc) break;
    if (verbose)
      std::fprintf(stderr,
                   "qmc_plan_tune: shifts_per_launch=%d smem_acc=%d min_ctas=%d imm_shifts=%d ctas=%d specialised=%d: "
                   "%.4f ms\n",
                   cd.mc, cd.smacc, cd.minb, cd.imm, trial.nblk,
                   (!trial.launches.empty() && trial.launches[0].cufunc) ? 1 : 0, tot / 3.0f);
    if (tot < best) {
      best = tot;
      best_c = cd;
    }
  }
  cudaFree(dres);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  if (best_c.mc != pl->mc || best_c.smacc != pl->tune.smacc || best_c.minb != pl->tune.minb ||
      best_c.imm != pl->imm) {
    TuneChoice tc = pl->tune;
    tc.mc = best_c.mc;
    tc.smacc = best_c.smacc;
    tc.minb = best_c.minb;
    tc.imm = best_c.imm;
    Plan fresh;
    rc = plan_build(&fresh, sp.d, sp.n, sp.m, sp.g.data(), sp.shifts.data(), sp.t, &sp.f, tc);
    if (rc) return rc;
    rc = plan_alloc(&fresh, nullptr, false);
    if (rc) return rc;
    cudaDeviceSynchronize();
    plan_free(pl, nullptr);
    fresh.saved = std::move(pl->saved);
    fresh.ev_before = pl->ev_before;
    fresh.ev_after = pl->ev_after;
    *pl = std::move(fresh);
  }
  if (shifts_per_launch_out) *shifts_per_launch_out = pl->mc;
  return QMC_OK;
}

int qmc_plan_execute(qmc_plan plan, qmc_result* out, double* per_shift, void* stream) {
  if (!plan) return fail(QMC_EINVAL, "null plan");
  return plan_execute(reinterpret_cast<Plan*>(plan), out, per_shift, (cudaStream_t)stream);
}

int qmc_plan_destroy(qmc_plan plan) {
  if (!plan) return QMC_OK;
  Plan* pl = reinterpret_cast<Plan*>(plan);
  cudaDeviceSynchronize();
  plan_free(pl, nullptr);
  delete pl;
  return QMC_OK;
}

int qmc_plan_launches(qmc_plan plan, int32_t* launches_out) {
  if (!plan || !launches_out) return fail(QMC_EINVAL, "null argument");
  *launches_out = (int32_t)reinterpret_cast<Plan*>(plan)->launches.size() + 1;
  return QMC_OK;
}

int qmc_integrate_to_tolerance(int32_t d, int32_t levels, const uint64_t* n, const uint64_t* g, int32_t m,
                               const double* shifts, qmc_transform t, const qmc_integrand* f, double rel_tol,
                               qmc_result* out, int32_t* level_out, void* stream) {
  if (levels < 1 || levels > 64 || !n || !g || !out || !(rel_tol > 0.0)) return fail(QMC_EINVAL, "bad ladder arguments");
  if (is_device_pointer(out)) return fail(QMC_EINVAL, "the result must be host memory");
  int rc = QMC_OK;
  for (int l = 0; l < levels; ++l) {
    rc = qmc_integrate(d, n[l], m, g + (size_t)l * d, shifts, t, f, out, nullptr, stream);
    if (rc != QMC_OK && rc != QMC_ENONFINITE && rc != QMC_EDEFORM) return rc;
    if (level_out) *level_out = l;
    const double mag = std::hypot(out->mean[0], out->mean[1]);
    const double err = std::hypot(out->err[0], out->err[1]);
    if (mag > 0.0 && err <= rel_tol * mag) return rc;
  }
  out->status = QMC_ETIMEOUT;
  return fail(QMC_ETIMEOUT, "relative error %.3g not reached after %d lattices", rel_tol, levels);
}

int qmc_integrate_extensible(int32_t d, int32_t log2_n0, int32_t levels, const uint64_t* g, int32_t m,
                             const double* shifts, qmc_transform t, const qmc_integrand* f, double rel_tol,
                             qmc_result* out, double* per_shift, int32_t* level_out, void* stream) {
  if (levels < 1 || log2_n0 < 1 || log2_n0 + levels - 1 > 30 || !g || !shifts || !out || !(rel_tol > 0.0) ||
      m < 2 || d < 1 || d > QMC_DMAX)
    return fail(QMC_EINVAL, "bad extensible-lattice arguments");
  if (is_device_pointer(out) || (per_shift && is_device_pointer(per_shift)))
    return fail(QMC_EINVAL, "the results must be host memory");
  for (int i = 0; i < d; ++i)
    if ((g[i] & 1) == 0) return fail(QMC_EINVAL, "g[%d] must be odd (a unit modulo every power of two)", i);
  std::vector<double> q((size_t)m * 2), qn((size_t)m * 2), sh2((size_t)m * d);
  std::vector<uint64_t> gl(d);
  int rc = QMC_OK;
  uint64_t nonfinite = 0, deform = 0;
  for (int l = 0; l < levels; ++l) {
    const uint64_t n = 1ull << (log2_n0 + (l == 0 ? 0 : l - 1));  // the size of the rule evaluated at this level
    for (int i = 0; i < d; ++i) gl[i] = g[i] % n == 0 ? 1 : g[i] % n;  // n = 2: every odd g is 1
    const double* sh = shifts;
    if (l > 0) {
      // the points of size 2n that are not in size n: the size-n lattice shifted by g / (2n)
      const double two_n = (double)(2 * n);
      for (int k = 0; k < m; ++k)
        for (int i = 0; i < d; ++i) {
          double v = shifts[(size_t)k * d + i] + (double)(g[i] % (2 * n)) / two_n;
          sh2[(size_t)k * d + i] = v >= 1.0 ? v - 1.0 : v;
        }
      sh = sh2.data();
    }
    qmc_result r;
    rc = qmc_integrate(d, n, m, gl.data(), sh, t, f, &r, l == 0 ? q.data() : qn.data(), stream);
    if (rc != QMC_OK && rc != QMC_ENONFINITE && rc != QMC_EDEFORM) return rc;
    if (l > 0)
      for (size_t u = 0; u < q.size(); ++u) q[u] = 0.5 * (q[u] + qn[u]);
    nonfinite += r.nonfinite;
    deform += r.deform_violations;
    rc = qmc_combine_shifts(m, q.data(), out);  // Eq. (3) on the per-shift values of size 2^(log2_n0 + l)
    if (rc) return rc;
    out->nonfinite = nonfinite;
    out->deform_violations = deform;
    out->status = nonfinite ? QMC_ENONFINITE : (deform ? QMC_EDEFORM : QMC_OK);
    if (level_out) *level_out = l;
    if (per_shift) std::memcpy(per_shift, q.data(), q.size() * sizeof(double));
    const double mag = std::hypot(out->mean[0], out->mean[1]);
    const double err = std::hypot(out->err[0], out->err[1]);
    if (mag > 0.0 && err <= rel_tol * mag) return out->status;
  }
  out->status = QMC_ETIMEOUT;
  return fail(QMC_ETIMEOUT, "relative error %.3g not reached by n = 2^%d", rel_tol, log2_n0 + levels - 1);
}

int qmc_combine_shifts(int32_t m, const double* per_shift, qmc_result* out) {
  if (m < 2 || !per_shift || !out) return fail(QMC_EINVAL, "combine needs m >= 2 values and an output");
  std::memset(out, 0, sizeof(*out));
  for (int part = 0; part < 2; ++part) {
    // Neumaier-compensated two-pass mean and variance
    double s = 0.0, c = 0.0;
    for (int k = 0; k < m; ++k) {
      const double v = per_shift[2 * k + part], t = s + v;
      c += std::fabs(s) >= std::fabs(v) ? (s - t) + v : (v - t) + s;
      s = t;
    }
    const double mean = (s + c) / (double)m;
    double vs = 0.0, vc = 0.0;
    for (int k = 0; k < m; ++k) {
      const double dlt = per_shift[2 * k + part] - mean, v = dlt * dlt, t = vs + v;
      vc += std::fabs(vs) >= std::fabs(v) ? (vs - t) + v : (v - t) + vs;
      vs = t;
    }
    out->mean[part] = mean;
    out->var[part] = (vs + vc) / ((double)m * (double)(m - 1));
    out->err[part] = std::sqrt(out->var[part]);
  }
  out->status = QMC_OK;
  return QMC_OK;
}

int qmc_plan_describe(qmc_plan plan, char* buf, int32_t len) {
  if (!plan || !buf || len < 1) return fail(QMC_EINVAL, "null plan or buffer");
  const Plan* pl = reinterpret_cast<const Plan*>(plan);
  const Launch* ln = pl->launches.empty() ? nullptr : &pl->launches[0];
  int L = 0;
  if (ln && ln->params.size() >= sizeof(RuleParams<float>)) {
    int32_t v;
    std::memcpy(&v, ln->params.data() + offsetof(RuleParams<float>, L), sizeof(v));
    L = v;
  }
  snprintf(buf, (size_t)len,
           "d=%d n=%llu m=%d complex=%d orders=%d shifts_per_launch=%d launches=%zu specialised=%d ctas=%d L=%d "
           "smem_acc=%d min_ctas=%d imm_shifts=%d",
           pl->d, (unsigned long long)pl->n, pl->m, pl->is_complex, pl->orders, pl->mc, pl->launches.size() + 1,
           (ln && ln->cufunc) ? 1 : 0, pl->nblk, L, (ln && ln->smem) ? 1 : 0, pl->tune.minb,
           (ln && ln->cufunc) ? pl->imm : 0);
  return QMC_OK;
}

int qmc_plan_record_events(qmc_plan plan, void* before_rule, void* after_rule) {
  if (!plan) return fail(QMC_EINVAL, "null plan");
  Plan* pl = reinterpret_cast<Plan*>(plan);
  pl->ev_before = (cudaEvent_t)before_rule;
  pl->ev_after = (cudaEvent_t)after_rule;
  return QMC_OK;
}

int qmc_integrate(int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts, qmc_transform t,
                  const qmc_integrand* f, qmc_result* out, double* per_shift, void* stream) {
  Plan pl;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = plan_build(&pl, d, n, m, g, shifts, t, f, TuneChoice{});
  if (rc) return rc;
  rc = plan_alloc(&pl, s, true);
  if (rc) return rc;
  rc = plan_execute(&pl, out, per_shift, s);
  plan_free(&pl, s);
  return rc;
}

// Evaluates listed (j, k) terms with the kernels of a built plan; each sample
// gets `vstride` values (2: real and imaginary part; epsilon plans: one per order).
static int sample_with_plan(Plan& pl, int32_t d, int32_t count, const uint64_t* j, const int32_t* k, double* values,
                            int vstride, uint64_t* idx, double* coord, cudaStream_t st) {
  const int dd = d;
  // group samples by shift chunk (each launch holds mc shifts)
  std::vector<std::vector<int>> by_chunk(pl.launches.size());
  for (int s = 0; s < count; ++s) by_chunk[k[s] / pl.mc].push_back(s);
  size_t bytes = (size_t)count * (8 + 4 + 8 * vstride + 8 * dd + 8 * dd) + 64;
  char* dbuf = nullptr;
  QMC_CUDA(cudaMallocAsync((void**)&dbuf, bytes, st));
  uint64_t* dj = (uint64_t*)dbuf;
  int32_t* dk = (int32_t*)(dj + count);
  double* dv = (double*)(((uintptr_t)(dk + count) + 15) & ~(uintptr_t)15);
  uint64_t* di = (uint64_t*)(dv + (size_t)vstride * count);
  double* dc = (double*)(di + (size_t)count * dd);
  std::vector<uint64_t> hj(count);
  std::vector<int32_t> hk(count);
  std::vector<int> order;
  for (size_t c = 0; c < by_chunk.size(); ++c)
    for (int s : by_chunk[c]) order.push_back(s);
  for (int q = 0; q < count; ++q) {
    hj[q] = j[order[q]];
    hk[q] = k[order[q]] % pl.mc;
  }
  QMC_CUDA(cudaMemcpyAsync(dj, hj.data(), 8 * (size_t)count, cudaMemcpyHostToDevice, st));
  QMC_CUDA(cudaMemcpyAsync(dk, hk.data(), 4 * (size_t)count, cudaMemcpyHostToDevice, st));
  int off = 0;
  for (size_t c = 0; c < by_chunk.size(); ++c) {
    int cnt = (int)by_chunk[c].size();
    if (!cnt) continue;
    SampleIO sio;
    sio.count = cnt;
    sio.stride = vstride;
    sio.j = dj + off;
    sio.k = dk + off;
    sio.values = dv + (size_t)vstride * off;
    sio.idx = di + (size_t)off * dd;
    sio.coord = dc + (size_t)off * dd;
    const Launch& ln = pl.launches[c];
    void* args[4];
    double* partial = nullptr;
    unsigned long long* counters = nullptr;
    args[0] = (void*)ln.params.data();
    args[1] = &partial;
    args[2] = &counters;
    args[3] = &sio;
    int rc = launch_any(ln, dim3((cnt + 255) / 256), args, st);
    if (rc) return rc;
    off += cnt;
  }
  std::vector<double> hv((size_t)vstride * count), hc((size_t)count * dd);
  std::vector<uint64_t> hi((size_t)count * dd);
  QMC_CUDA(cudaMemcpyAsync(hv.data(), dv, 8 * (size_t)vstride * count, cudaMemcpyDeviceToHost, st));
  QMC_CUDA(cudaMemcpyAsync(hi.data(), di, 8 * (size_t)count * dd, cudaMemcpyDeviceToHost, st));
  QMC_CUDA(cudaMemcpyAsync(hc.data(), dc, 8 * (size_t)count * dd, cudaMemcpyDeviceToHost, st));
  QMC_CUDA(cudaFreeAsync(dbuf, st));
  QMC_CUDA(cudaStreamSynchronize(st));
  for (int q = 0; q < count; ++q) {
    int s = order[q];
    for (int v = 0; v < vstride; ++v) values[(size_t)vstride * s + v] = hv[(size_t)vstride * q + v];
    for (int i = 0; i < dd; ++i) {
      if (idx) idx[(size_t)s * dd + i] = hi[(size_t)q * dd + i];
      if (coord) coord[(size_t)s * dd + i] = hc[(size_t)q * dd + i];
    }
  }
  return QMC_OK;
}

static int check_samples(uint64_t n, int32_t m, int32_t count, const uint64_t* j, const int32_t* k,
                         const double* values) {
  if (count < 0 || (count > 0 && (!j || !k || !values))) return fail(QMC_EINVAL, "bad sample arrays");
  for (int s = 0; s < count; ++s) {
    if (j[s] >= n) return fail(QMC_EINVAL, "sample %d: j=%llu >= n", s, (unsigned long long)j[s]);
    if (k[s] < 0 || k[s] >= m) return fail(QMC_EINVAL, "sample %d: k=%d outside [0, m)", s, k[s]);
  }
  return QMC_OK;
}

int qmc_sample_points(int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts, qmc_transform t,
                      const qmc_integrand* f, int32_t count, const uint64_t* j, const int32_t* k, double* values,
                      uint64_t* idx, double* coord, void* stream) {
  int rc = check_samples(n, m, count, j, k, values);
  if (rc || count == 0) return rc;
  Plan pl;
  rc = plan_build(&pl, d, n, m, g, shifts, t, f, TuneChoice{});
  if (rc) return rc;
  return sample_with_plan(pl, d, count, j, k, values, 2, idx, coord, (cudaStream_t)stream);
}

int qmc_eps_plan_create(int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts, qmc_transform t,
                        const qmc_integrand* f, const qmc_eps* eps, qmc_plan* plan_out) {
  if (!plan_out || !eps) return fail(QMC_EINVAL, "null plan_out or epsilon descriptor");
  *plan_out = nullptr;
  std::unique_ptr<Plan> pl(new Plan());
  int rc = plan_build(pl.get(), d, n, m, g, shifts, t, f, TuneChoice{}, eps);
  if (rc) return rc;
  rc = plan_alloc(pl.get(), nullptr, false);
  if (rc) return rc;
  pl->saved.save(d, n, m, g, shifts, t, f);
  pl->saved.eps = *eps;
  *plan_out = reinterpret_cast<qmc_plan>(pl.release());
  return QMC_OK;
}

int qmc_integrate_eps(int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts, qmc_transform t,
                      const qmc_integrand* f, const qmc_eps* eps, qmc_result* out, double* per_shift, void* stream) {
  if (!eps) return fail(QMC_EINVAL, "null epsilon descriptor");
  Plan pl;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = plan_build(&pl, d, n, m, g, shifts, t, f, TuneChoice{}, eps);
  if (rc) return rc;
  rc = plan_alloc(&pl, s, true);
  if (rc) return rc;
  rc = plan_execute(&pl, out, per_shift, s);
  plan_free(&pl, s);
  return rc;
}

int qmc_sample_points_eps(int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts,
                          qmc_transform t, const qmc_integrand* f, const qmc_eps* eps, int32_t count,
                          const uint64_t* j, const int32_t* k, double* values, void* stream) {
  if (!eps) return fail(QMC_EINVAL, "null epsilon descriptor");
  int rc = check_samples(n, m, count, j, k, values);
  if (rc || count == 0) return rc;
  Plan pl;
  rc = plan_build(&pl, d, n, m, g, shifts, t, f, TuneChoice{}, eps);
  if (rc) return rc;
  return sample_with_plan(pl, d, count, j, k, values, eps->orders, nullptr, nullptr, (cudaStream_t)stream);
}

}  // extern "C"

namespace qmc {
template void fill_common<float>(RuleParams<float>&, int32_t, uint64_t, const uint64_t*, const qmc_transform&,
                                 const qmc_integrand*);
template void fill_common<double>(RuleParams<double>&, int32_t, uint64_t, const uint64_t*, const qmc_transform&,
                                  const qmc_integrand*);
}  // namespace qmc

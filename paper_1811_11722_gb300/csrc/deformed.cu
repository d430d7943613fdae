// Plan builder for contour-deformed (complex) sector integrands.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "deformed.cuh"
#include "plan.h"

namespace qmc {

// QMC_DEFORMED_PACKED=0 keeps FP32 plans on the one-shift kernel.
static bool deformed_packed_enabled() {
  const char* e = std::getenv("QMC_DEFORMED_PACKED");
  return !(e && e[0] == '0');
}

// The packed FP32 variant (two shifts per instruction), d <= kDef2DMax.
static const void* deformed2_ptr(int d) {
  switch (d) {
    case 1: return (const void*)&deformed2_kernel<1>;
    case 2: return (const void*)&deformed2_kernel<2>;
    case 3: return (const void*)&deformed2_kernel<3>;
    case 4: return (const void*)&deformed2_kernel<4>;
    case 5: return (const void*)&deformed2_kernel<5>;
    default: return nullptr;
  }
}

constexpr int kMcDef = 8;  // shifts per launch (matches the kernel's shared accumulators)

// Offset of q_ij (i <= j) in the nested degree-2 layout (host copy of q_off).
static int q_off_host(int D, int i, int j) {
  int off = 1;
  for (int a = 0; a < i; ++a) off += 1 + (D - a);
  return off + 1 + (j - i);
}

template <typename R>
static int build_def(Plan* pl, int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts,
                     const qmc_transform& t, const qmc_integrand* f, const TuneChoice& tune) {
  if (d > kDFast) return fail(QMC_EUNSUPPORTED, "deformed sector integrands need d <= %d", kDFast);
  RuleParams<R> base;
  fill_common(base, d, n, g, t, f);
  auto cf = pack_dense(f->F, d, 2);
  // J = I + i M with M_kl = -lam (y_k (1 - y_k) S_kl + delta_kl (1 - 2 y_k) dF_k), S = Hessian of F.
  // |J_kk| >= 1 and sum_{l != k} |M_kl| <= lam / 4 * sum_{l != k} |S_kl|: below 1 for every row,
  // J is strictly row diagonally dominant on the whole cube and LU needs no pivoting.
  double worst = 0.0;
  for (int k = 0; k < d; ++k) {
    double row = 0.0;
    for (int l = 0; l < d; ++l) {
      if (l == k) continue;
      const int a = k < l ? k : l, b = k < l ? l : k;
      row += std::fabs(cf[q_off_host(d, a, b)]);
    }
    worst = std::max(worst, 0.25 * f->lambda * row);
  }
  const bool fast = worst < 1.0 && t.kind == QMC_TRANSFORM_KOROBOV && t.alpha == 3 && !tune.force_general;
  const bool u_linear = poly_degree(f->U, d) <= 1;  // U on its degree-1 slots only
  // FP32 with two shifts per instruction: the FAST variant, U^-2 F^-1, d <= kDef2DMax
  const bool packed = sizeof(R) == 4 && fast && u_linear && d <= kDef2DMax && f->aU == -2 && f->aF == -1 &&
                      deformed_packed_enabled();
  const void* func = nullptr;
  switch (d) {
#define QMC_D_CASE(DD) \
  case DD:             \
    func = deformed_ptr<R, DD>(fast, u_linear); \
    break;
    QMC_D_CASE(1) QMC_D_CASE(2) QMC_D_CASE(3) QMC_D_CASE(4) QMC_D_CASE(5) QMC_D_CASE(6) QMC_D_CASE(7)
    QMC_D_CASE(8)
#undef QMC_D_CASE
    default: break;
  }
  if (packed) func = deformed2_ptr(d);
  if (!func) return fail(QMC_EUNSUPPORTED, "no deformed kernel for d=%d", d);
  auto cu = pack_dense(f->U, d, u_linear ? 1 : 2);
  for (size_t i = 0; i < cu.size(); ++i) base.cU[i] = (R)cu[i];
  for (size_t i = 0; i < cf.size(); ++i) base.cF[i] = (R)cf[i];
  for (int k = 0; k < d; ++k)  // -lambda d2F/dy_k dy_l (constant: F has degree 2)
    for (int l = 0; l < d; ++l) {
      const int a = k < l ? k : l, b = k < l ? l : k;
      const double h = (k == l ? 2.0 : 1.0) * cf[q_off_host(d, a, b)];
      base.cF[kDefHessOff + k * d + l] = (R)(-f->lambda * h);
    }
  if (packed) {  // (c, c) pairs: U's linear slots, F's slots, then the Hessian of F, k-major
    int o = 0;
    for (size_t i = 0; i < cu.size(); ++i, ++o) base.cp[o] = make_float2((float)cu[i], (float)cu[i]);
    for (size_t i = 0; i < cf.size(); ++i, ++o) base.cp[o] = make_float2((float)cf[i], (float)cf[i]);
    for (int k = 0; k < d; ++k)
      for (int l = 0; l < d; ++l, ++o) {
        const int a = k < l ? k : l, b = k < l ? l : k;
        const float h = (float)((k == l ? 2.0 : 1.0) * cf[q_off_host(d, a, b)]);
        base.cp[o] = make_float2(h, h);
      }
    if (o > kPairCoefMax) return fail(QMC_EUNSUPPORTED, "deformed: %d coefficient pairs", o);
  }
  // Transform weight constants.  FP64 normalises each factor in the kernel.
  // FP32 FAST multiplies the factors u and cubes the product: (2a+1)!/(a!)^2
  // = 140 per dimension remains; other FP32 Korobov plans raise the product of
  // the factors 4u to the power alpha: ((2a+1)!/(a!)^2 / 4^a) per dimension.
  base.value_scale = 1.0;
  if (sizeof(R) == 4 && base.tr == TR_KOROBOV)
    base.value_scale = fast ? std::pow((double)base.kor[7], (double)d)
                            : std::pow((double)base.kor[7] / std::pow(4.0, (double)base.alpha), (double)d);
  base.check_finite = 1;
  int nblk = 0, L = 0, occ = 0;
  uint64_t tiles = 0;
  int rc = grid_occupancy(func, 0, tune.occupancy, occ);
  if (rc) return rc;
  rc = grid_shape(occ, n, 0, tune.L, nblk, L, tiles);
  if (rc) return rc;
  pl->param_kind = sizeof(R) == 4 ? 1 : 2;
  pl->grid_occ = occ;
  pl->grid_capped = false;  // one resident wave whatever the caller's cap
  base.L = L;
  base.tiles = tiles;
  base.nblk = nblk;
  pl->nblk = nblk;
  pl->func = func;
  pl->mc = kMcDef;
  pl->final_scale = base.value_scale;
  pl->is_complex = 1;
  for (int k0 = 0; k0 < m; k0 += kMcDef) {
    const int mk = std::min(kMcDef, m - k0);
    RuleParams<R> P = base;
    P.m_launch = mk;
    P.k_base = k0;
    for (int kk = 0; kk < mk; ++kk)
      for (int i = 0; i < d; ++i) {
        uint64_t s64 = shift_fixed64(shifts[(size_t)(k0 + kk) * d + i]);
        set_shift(P, kk, i, s64);
      }
    Launch ln;
    ln.func = func;
    ln.grid = dim3(nblk);
    ln.params.resize(sizeof(P));
    std::memcpy(ln.params.data(), &P, sizeof(P));
    pl->launches.push_back(std::move(ln));
  }
  return QMC_OK;
}

int build_deformed_plan(Plan* pl, int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts,
                        const qmc_transform& t, const qmc_integrand* f, const TuneChoice& tune) {
  if (f->precision == QMC_FP32EVAL) return build_def<float>(pl, d, n, m, g, shifts, t, f, tune);
  return build_def<double>(pl, d, n, m, g, shifts, t, f, tune);
}

}  // namespace qmc

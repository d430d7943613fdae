// Lookup of kernel instantiations by their runtime description.  Each getter
// returns the address of a __global__ function (for cudaLaunchKernel) or null
// when no specialisation exists for the request.
#pragma once

#include <cstdint>

#include "qmc_internal.h"

namespace qmc {

// Dense sector kernel, U of degree ku, F of degree kf, d = D <= kDFast.
// One explicit specialisation per (precision, D), each in its own unit.
// Only U^-2 F^-1; check selects the NaN/Inf-counting variant.
template <typename R, int D>
const void* sector_ptr(int mc, int tr, int alpha, int ku, int kf, bool check);
#define QMC_DECL_SECTOR(R, D) template <> const void* sector_ptr<R, D>(int, int, int, int, int, bool);
QMC_DECL_SECTOR(float, 1) QMC_DECL_SECTOR(float, 2) QMC_DECL_SECTOR(float, 3) QMC_DECL_SECTOR(float, 4)
QMC_DECL_SECTOR(float, 5) QMC_DECL_SECTOR(float, 6) QMC_DECL_SECTOR(float, 7) QMC_DECL_SECTOR(float, 8)
QMC_DECL_SECTOR(double, 1) QMC_DECL_SECTOR(double, 2) QMC_DECL_SECTOR(double, 3) QMC_DECL_SECTOR(double, 4)
QMC_DECL_SECTOR(double, 5) QMC_DECL_SECTOR(double, 6) QMC_DECL_SECTOR(double, 7) QMC_DECL_SECTOR(double, 8)
#undef QMC_DECL_SECTOR

// Epsilon-order kernel (Eq. 7 expansion): dense U of degree 1, F of degree 2,
// U^-2 F^-1 at eps = 0, d = D, baker or Korobov-3; ne = 3 or kEpsMax orders
// accumulated (kEpsAcc / ne shifts per launch).
template <typename R, int D>
const void* eps_ptr(int ne, int tr);
#define QMC_DECL_EPS(R, D) template <> const void* eps_ptr<R, D>(int, int);
QMC_DECL_EPS(float, 1) QMC_DECL_EPS(float, 2) QMC_DECL_EPS(float, 3) QMC_DECL_EPS(float, 4)
QMC_DECL_EPS(float, 5) QMC_DECL_EPS(float, 6) QMC_DECL_EPS(float, 7) QMC_DECL_EPS(float, 8)
QMC_DECL_EPS(double, 1) QMC_DECL_EPS(double, 2) QMC_DECL_EPS(double, 3) QMC_DECL_EPS(double, 4)
QMC_DECL_EPS(double, 5) QMC_DECL_EPS(double, 6) QMC_DECL_EPS(double, 7) QMC_DECL_EPS(double, 8)
#undef QMC_DECL_EPS

// Contour-deformed complex sector kernel, d = D <= kDFast: fast = Korobov 3
// and unpivoted LU (host-checked dominance); otherwise runtime transform and
// pivoted LU.
template <typename R, int D>
const void* deformed_ptr(bool fast, bool u_linear);
// Deformed sector kernels: the Hessian of F times -lambda, [k][l] with row
// stride d, kept in RuleParams::cF after F's nested-Horner slots.
constexpr int kDefHessOff = 64;
static_assert(kDefHessOff >= poly_slots(kDFast, 2) && kDefHessOff + kDFast * kDFast <= kPolyCoefMax,
              "deformed Hessian table placement");
#define QMC_DECL_DEF(R, D) template <> const void* deformed_ptr<R, D>(bool, bool);
QMC_DECL_DEF(float, 1) QMC_DECL_DEF(float, 2) QMC_DECL_DEF(float, 3) QMC_DECL_DEF(float, 4)
QMC_DECL_DEF(float, 5) QMC_DECL_DEF(float, 6) QMC_DECL_DEF(float, 7) QMC_DECL_DEF(float, 8)
QMC_DECL_DEF(double, 1) QMC_DECL_DEF(double, 2) QMC_DECL_DEF(double, 3) QMC_DECL_DEF(double, 4)
QMC_DECL_DEF(double, 5) QMC_DECL_DEF(double, 6) QMC_DECL_DEF(double, 7) QMC_DECL_DEF(double, 8)
#undef QMC_DECL_DEF

// Separable integrands (const / separable exp / trig), runtime d and
// Korobov weight (factors normalised, value scale 1).
template <typename R>
const void* separable_ptr_t(int tr, int fk);
template <> const void* separable_ptr_t<float>(int tr, int fk);
template <> const void* separable_ptr_t<double>(int tr, int fk);
inline const void* separable_ptr(bool fp32, int tr, int fk) {
  return fp32 ? separable_ptr_t<float>(tr, fk) : separable_ptr_t<double>(tr, fk);
}

// General sparse-polynomial sector kernel, runtime d, transform and powers.
template <typename R>
const void* general_ptr_t();
template <> const void* general_ptr_t<float>();
template <> const void* general_ptr_t<double>();
inline const void* general_ptr(bool fp32) { return fp32 ? general_ptr_t<float>() : general_ptr_t<double>(); }

// General sparse kernel with kEpsMax epsilon orders (kEpsAcc / kEpsMax shifts per launch).
template <typename R>
const void* general_eps_ptr_t();
template <> const void* general_eps_ptr_t<float>();
template <> const void* general_eps_ptr_t<double>();
inline const void* general_eps_ptr(bool fp32) {
  return fp32 ? general_eps_ptr_t<float>() : general_eps_ptr_t<double>();
}

// Final deterministic pass: per-shift sums -> Q^(k), Qbar, sigma^2; the
// batched form takes a device array of FinalizeArgs, one CTA per problem.
const void* finalize_ptr();
const void* finalize_batch_ptr();
const void* persist_kernel_ptr();  // batched sectors in one persistent launch (persist.cu)

// Arguments of the final pass.
struct FinalizeArgs {
  const double* partial;   // [groups][m][nblk][2]
  int32_t nblk;
  int32_t m;
  int32_t is_complex;
  int32_t groups;          // finalize_kernel: CTA b finalises group b (epsilon order b, integrand b)
  int32_t sum_last;        // 1: the last group is the sum of the others (shared-lattice plans)
  int32_t pad;
  double dn;      // n as a double
  double value_scale;
  double offset[2];  // added to Q^(k) of each part (control-variate integral)
  unsigned long long* counters;  // [groups][2], reset to zero after reading
  qmc_result* result;            // device [groups]
  double* per_shift;             // device [groups][m][2] or null
};

}  // namespace qmc

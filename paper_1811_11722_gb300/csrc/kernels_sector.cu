// Instantiations of the specialised sector, epsilon-order and deformed kernels for one
// (precision, d).
// Compiled once per pair with -DQMC_REAL=float|double -DQMC_D=1..8 so the
// build spreads the template work over parallel nvcc processes.
#include "kernel_table.h"
#include "deformed.cuh"
#include "rule_kernels.cuh"

#ifndef QMC_REAL
#error "QMC_REAL must be float or double"
#endif
#ifndef QMC_D
#error "QMC_D must be 1..8"
#endif

namespace qmc {

#define QMC_SECTOR_CK(R, MC, TR, AL, KU, KF)                                                   \
  do {                                                                                         \
    if (check) return (const void*)&sector_kernel<R, QMC_D, MC, TR, AL, KU, KF, true>;         \
    return (const void*)&sector_kernel<R, QMC_D, MC, TR, AL, KU, KF, false>;                   \
  } while (0)
#define QMC_SECTOR_TR(R, MC, KU, KF)                                              \
  do {                                                                            \
    if (tr == TR_NONE) QMC_SECTOR_CK(R, MC, TR_NONE, 0, KU, KF);                  \
    if (tr == TR_BAKER) QMC_SECTOR_CK(R, MC, TR_BAKER, 0, KU, KF);                \
    if (tr == TR_KOROBOV && alpha == 3) QMC_SECTOR_CK(R, MC, TR_KOROBOV, 3, KU, KF); \
  } while (0)

template <>
const void* sector_ptr<QMC_REAL, QMC_D>(int mc, int tr, int alpha, int ku, int kf, bool check) {
  // FP32 is FMA-pipe bound: shift-chunk sizes 8/16/32 trade registers for
  // reuse of the per-point index work.  FP64 is DP-pipe bound on this part
  // and takes one chunk size.
  constexpr bool kF32 = sizeof(QMC_REAL) == 4;
  if (ku == 1 && kf == 2) {
    if constexpr (kF32) {
      if (mc == 8) QMC_SECTOR_TR(QMC_REAL, 8, 1, 2);
      if (mc == 32) QMC_SECTOR_TR(QMC_REAL, 32, 1, 2);
    }
    if (mc == 16) QMC_SECTOR_TR(QMC_REAL, 16, 1, 2);
  }
  if constexpr (kF32) {
    if (ku == 2 && kf == 3 && mc == 16) QMC_SECTOR_TR(QMC_REAL, 16, 2, 3);
  }
  return nullptr;
}

template <>
const void* eps_ptr<QMC_REAL, QMC_D>(int ne, int tr) {
  // orders x shifts per launch = kEpsAcc accumulators
  if (ne == 3) {
    if (tr == TR_BAKER) return (const void*)&eps_kernel<QMC_REAL, QMC_D, kEpsAcc / 3, 3, TR_BAKER, 0>;
    if (tr == TR_KOROBOV) return (const void*)&eps_kernel<QMC_REAL, QMC_D, kEpsAcc / 3, 3, TR_KOROBOV, 3>;
  }
  if (ne == kEpsMax) {
    if (tr == TR_BAKER) return (const void*)&eps_kernel<QMC_REAL, QMC_D, kEpsAcc / kEpsMax, kEpsMax, TR_BAKER, 0>;
    if (tr == TR_KOROBOV) return (const void*)&eps_kernel<QMC_REAL, QMC_D, kEpsAcc / kEpsMax, kEpsMax, TR_KOROBOV, 3>;
  }
  return nullptr;
}

template <>
const void* deformed_ptr<QMC_REAL, QMC_D>(bool fast, bool u_linear) {
  if (u_linear)
    return fast ? (const void*)&deformed_kernel<QMC_REAL, QMC_D, true, 1>
                : (const void*)&deformed_kernel<QMC_REAL, QMC_D, false, 1>;
  return fast ? (const void*)&deformed_kernel<QMC_REAL, QMC_D, true, 2>
              : (const void*)&deformed_kernel<QMC_REAL, QMC_D, false, 2>;
}

}  // namespace qmc

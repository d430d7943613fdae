// Separable and general rule kernels for one precision (compiled once per
// precision with -DQMC_REAL=float|double).
#include "kernel_table.h"
#include "rule_kernels.cuh"

#ifndef QMC_REAL
#error "QMC_REAL must be float or double"
#endif

namespace qmc {

#define QMC_SEP_FK(R, TR, AL)                                                        \
  do {                                                                               \
    if (fk == FK_CONST) return (const void*)&separable_kernel<R, 8, TR, FK_CONST>;   \
    if (fk == FK_SEPEXP) return (const void*)&separable_kernel<R, 8, TR, FK_SEPEXP>; \
    if (fk == FK_TRIG) return (const void*)&separable_kernel<R, 8, TR, FK_TRIG>;     \
  } while (0)

template <>
const void* separable_ptr_t<QMC_REAL>(int tr, int fk) {
  if (tr == TR_NONE) QMC_SEP_FK(QMC_REAL, TR_NONE, 0);
  if (tr == TR_BAKER) QMC_SEP_FK(QMC_REAL, TR_BAKER, 0);
  if (tr == TR_KOROBOV) QMC_SEP_FK(QMC_REAL, TR_KOROBOV, 0);
  return nullptr;
}

template <>
const void* general_ptr_t<QMC_REAL>() {
  return (const void*)&general_kernel<QMC_REAL, 8>;
}

template <>
const void* general_eps_ptr_t<QMC_REAL>() {
  return (const void*)&general_eps_kernel<QMC_REAL>;
}

}  // namespace qmc

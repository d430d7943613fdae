// Control-variate kernels for one dimension (compiled with -DQMC_D=1..8).
#include "cv_device.cuh"
#include "cv_tc5.cuh"

#ifndef QMC_D
#error "QMC_D must be 1..8"
#endif

namespace qmc {

template <>
const void* cv_estimator_ptr<QMC_D>(int tr, int alpha) {
  if (tr == TR_BAKER) return (const void*)&cv_tc_kernel<QMC_D, TR_BAKER, 0>;
  if (tr == TR_KOROBOV && alpha == 3) return (const void*)&cv_tc_kernel<QMC_D, TR_KOROBOV, 3>;
  if (tr == TR_NONE) return (const void*)&cv_tc_kernel<QMC_D, TR_NONE, 0>;
  return nullptr;
}

template <>
const void* cv_estimator5_ptr<QMC_D>(int tr, int alpha) {
  if (tr == TR_BAKER) return (const void*)&cv_tc5_kernel<QMC_D, TR_BAKER, 0>;
  if (tr == TR_KOROBOV && alpha == 3) return (const void*)&cv_tc5_kernel<QMC_D, TR_KOROBOV, 3>;
  if (tr == TR_NONE) return (const void*)&cv_tc5_kernel<QMC_D, TR_NONE, 0>;
  return nullptr;
}

template <>
const void* cv_fit_ptr<QMC_D>() {
  return (const void*)&cv_fit_kernel<QMC_D>;
}

}  // namespace qmc

// Batched sectors: placeholder until the persistent batch kernel lands.
#include "plan.h"

using namespace qmc;

extern "C" {

int qmc_integrate_batch(int32_t count, const qmc_problem* problems, qmc_result* out, double* per_shift,
                        void* stream) {
  (void)count; (void)problems; (void)out; (void)per_shift; (void)stream;
  return fail(QMC_EUNSUPPORTED, "batched integration is not built yet");
}

int qmc_batch_plan_create(int32_t count, const qmc_problem* problems, qmc_batch_plan* plan_out) {
  (void)count; (void)problems;
  if (plan_out) *plan_out = nullptr;
  return fail(QMC_EUNSUPPORTED, "batched integration is not built yet");
}

int qmc_batch_plan_execute(qmc_batch_plan plan, qmc_result* out, double* per_shift, void* stream) {
  (void)plan; (void)out; (void)per_shift; (void)stream;
  return fail(QMC_EUNSUPPORTED, "batched integration is not built yet");
}

int qmc_batch_plan_destroy(qmc_batch_plan plan) {
  (void)plan;
  return QMC_OK;
}

}  // extern "C"

// Many independent rules (sectors of uneven dimension and point count) in one
// CUDA graph.
//
// Each problem keeps its own specialised kernel with its shifts and
// polynomial coefficients in the constant bank (kernel parameters), exactly
// as a single rule.  The graph holds one kernel node per (problem, shift
// chunk) with no edges between them, so the hardware scheduler runs the
// sectors side by side and back-fills SMs as small sectors finish, plus one
// batched final-pass node (one CTA per problem) that depends on all of them.
// The graph is built once per plan and replayed by every execute.
//
// Launch shape: a problem gets ceil(n m / W) CTAs (capped at one resident
// wave), W the evaluations per CTA; qmc_batch_plan_tune times a ladder of W
// on the device and keeps the fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <string>
#include <thread>
#include <cstring>
#include <memory>
#include <vector>

#include "plan.h"

namespace qmc {

struct BatchPlan {
  int count = 0;
  int total_m = 0;
  int max_m = 0;
  int launches = 0;
  uint64_t work_per_cta = 1ull << 20;
  std::vector<qmc_problem> src;          // host copy of the descriptors (pointers stay the caller's until create returns)
  std::vector<std::unique_ptr<Plan>> probs;
  std::vector<size_t> ps_off;            // per-shift offsets (doubles)
  void* ws = nullptr;
  qmc_result* res_dev = nullptr;
  double* ps_dev = nullptr;
  FinalizeArgs* fin_dev = nullptr;
  std::vector<FinalizeArgs> fin_host;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

static void batch_release(BatchPlan* bp) {
  if (bp->exec) cudaGraphExecDestroy(bp->exec);
  if (bp->graph) cudaGraphDestroy(bp->graph);
  bp->exec = nullptr;
  bp->graph = nullptr;
  if (bp->ws) cudaFree(bp->ws);
  bp->ws = nullptr;
}

// Validate and pack every problem; problem pointers are only read here.
static int batch_build(BatchPlan* bp, int32_t count, const qmc_problem* problems, uint64_t work_per_cta) {
  if (count < 1 || count > 65536) return fail(QMC_EINVAL, "batch count=%d outside [1, 65536]", count);
  if (!problems) return fail(QMC_EINVAL, "null problems");
  bp->count = count;
  bp->work_per_cta = work_per_cta;
  bp->probs.clear();
  bp->ps_off.clear();
  bp->total_m = 0;
  bp->max_m = 0;
  bp->launches = 1;
  int sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(QMC_ECUDA, "no CUDA device");
  }
  // pack every problem (and compile its specialised kernel) on the host
  // cores; problems are independent, the results keep the input order
  std::vector<std::unique_ptr<Plan>> plans(count);
  std::vector<int> rcs(count, QMC_OK);
  std::vector<std::string> errs(count);
  std::atomic<int> next{0};
  auto work = [&]() {
    int dev_here = 0;
    cudaSetDevice(dev);
    (void)dev_here;
    for (int i = next++; i < count; i = next++) {
      const qmc_problem& q = problems[i];
      std::unique_ptr<Plan> pl(new Plan());
      TuneChoice tc;
      const uint64_t evals = q.n * (uint64_t)std::max(q.m, 1);
      tc.max_ctas = (int)std::max<uint64_t>(1, std::min<uint64_t>((evals + work_per_cta - 1) / work_per_cta, 4ull * sms));
      rcs[i] = plan_build(pl.get(), q.d, q.n, q.m, q.g, q.shifts, q.t, q.f, tc);
      if (rcs[i]) errs[i] = qmc_last_error();
      plans[i] = std::move(pl);
    }
  };
  const unsigned nt = std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), (unsigned)std::min(count, 32)));
  std::vector<std::thread> th;
  for (unsigned t = 1; t < nt; ++t) th.emplace_back(work);
  work();
  for (auto& x : th) x.join();
  for (int i = 0; i < count; ++i) {
    if (rcs[i]) return fail(rcs[i], "problem %d: %s", i, errs[i].c_str());
    const Plan* pl = plans[i].get();
    bp->ps_off.push_back((size_t)bp->total_m * 2);
    bp->total_m += pl->m;
    bp->max_m = std::max(bp->max_m, pl->m);
    bp->launches += (int)pl->launches.size();
    bp->probs.push_back(std::move(plans[i]));
  }
  return QMC_OK;
}

static int batch_alloc(BatchPlan* bp) {
  size_t bytes = 0;
  std::vector<size_t> part_off(bp->count), cnt_off(bp->count);
  for (int i = 0; i < bp->count; ++i) {
    const Plan* pl = bp->probs[i].get();
    part_off[i] = bytes;
    bytes += (size_t)pl->m * pl->nblk * 2 * sizeof(double);
  }
  for (int i = 0; i < bp->count; ++i) {
    cnt_off[i] = bytes;
    bytes += 2 * sizeof(unsigned long long);
  }
  bytes = (bytes + 255) & ~(size_t)255;
  const size_t res_off = bytes;
  bytes += (size_t)bp->count * sizeof(qmc_result);
  bytes = (bytes + 255) & ~(size_t)255;
  const size_t ps_off = bytes;
  bytes += (size_t)bp->total_m * 2 * sizeof(double);
  bytes = (bytes + 255) & ~(size_t)255;
  const size_t fin_off = bytes;
  bytes += (size_t)bp->count * sizeof(FinalizeArgs);
  cudaError_t e = cudaMalloc(&bp->ws, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(QMC_ENOMEM, "batch workspace of %zu bytes: %s", bytes, cudaGetErrorString(e));
  }
  char* base = (char*)bp->ws;
  bp->res_dev = (qmc_result*)(base + res_off);
  bp->ps_dev = (double*)(base + ps_off);
  bp->fin_dev = (FinalizeArgs*)(base + fin_off);
  bp->fin_host.resize(bp->count);
  for (int i = 0; i < bp->count; ++i) {
    Plan* pl = bp->probs[i].get();
    pl->ws.partial = (double*)(base + part_off[i]);
    pl->ws.counters = (unsigned long long*)(base + cnt_off[i]);
    FinalizeArgs& A = bp->fin_host[i];
    std::memset(&A, 0, sizeof(A));
    A.partial = pl->ws.partial;
    A.nblk = pl->nblk;
    A.m = pl->m;
    A.is_complex = pl->is_complex;
    A.dn = (double)pl->n;
    A.value_scale = pl->final_scale;
    A.offset[0] = pl->offset[0];
    A.offset[1] = pl->offset[1];
    A.counters = pl->ws.counters;
    A.result = bp->res_dev + i;
    A.per_shift = bp->ps_dev + bp->ps_off[i];
  }
  e = cudaMemcpy(bp->fin_dev, bp->fin_host.data(), (size_t)bp->count * sizeof(FinalizeArgs), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "batch finalize descriptors");
  e = cudaMemset(base + cnt_off[0], 0, (size_t)bp->count * 2 * sizeof(unsigned long long));
  if (e != cudaSuccess) return cuda_fail(e, "batch counters");
  return QMC_OK;
}

static int batch_graph(BatchPlan* bp) {
  cudaError_t e = cudaGraphCreate(&bp->graph, 0);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
  std::vector<cudaGraphNode_t> nodes;
  SampleIO none;
  std::memset(&none, 0, sizeof(none));
  for (int i = 0; i < bp->count; ++i) {
    Plan* pl = bp->probs[i].get();
    for (Launch& ln : pl->launches) {
      double* partial = pl->ws.partial;
      unsigned long long* counters = pl->ws.counters;
      void* args[4] = {(void*)ln.params.data(), &partial, &counters, &none};
      cudaGraphNode_t node;
      int rc = graph_add_launch(bp->graph, ln, args, &node);
      if (rc) return rc;
      nodes.push_back(node);
    }
  }
  FinalizeArgs* fin = bp->fin_dev;
  void* fargs[1] = {&fin};
  cudaKernelNodeParams kp;
  std::memset(&kp, 0, sizeof(kp));
  kp.func = (void*)finalize_batch_ptr();
  kp.gridDim = dim3(bp->count);
  kp.blockDim = dim3(256);
  kp.sharedMemBytes = (unsigned)((size_t)bp->max_m * 2 * sizeof(double));
  kp.kernelParams = fargs;
  cudaGraphNode_t fnode;
  e = cudaGraphAddKernelNode(&fnode, bp->graph, nodes.data(), nodes.size(), &kp);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphAddKernelNode (final pass)");
  e = cudaGraphInstantiate(&bp->exec, bp->graph, 0);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  return QMC_OK;
}

static int batch_create(BatchPlan* bp, int32_t count, const qmc_problem* problems, uint64_t work_per_cta) {
  int rc = batch_build(bp, count, problems, work_per_cta);
  if (rc) return rc;
  rc = batch_alloc(bp);
  if (rc) return rc;
  return batch_graph(bp);
}

static int batch_execute(BatchPlan* bp, qmc_result* out, double* per_shift, cudaStream_t stream) {
  if (!out) return fail(QMC_EINVAL, "null result pointer");
  cudaError_t e = cudaGraphLaunch(bp->exec, stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  const bool out_dev = is_device_pointer(out);
  const bool ps_dev = per_shift ? is_device_pointer(per_shift) : true;
  const cudaMemcpyKind k_out = out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  e = cudaMemcpyAsync(out, bp->res_dev, (size_t)bp->count * sizeof(qmc_result), k_out, stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch results");
  if (per_shift) {
    e = cudaMemcpyAsync(per_shift, bp->ps_dev, (size_t)bp->total_m * 2 * sizeof(double),
                        ps_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch per-shift values");
  }
  if (!out_dev || !ps_dev) {
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch synchronise");
    if (!out_dev) {
      int worst = QMC_OK;
      for (int i = 0; i < bp->count; ++i)
        if (out[i].status != QMC_OK && worst == QMC_OK) worst = out[i].status;
      return worst;
    }
  }
  return QMC_OK;
}

}  // namespace qmc

using namespace qmc;

extern "C" {

int qmc_batch_plan_create(int32_t count, const qmc_problem* problems, qmc_batch_plan* plan_out) {
  if (!plan_out) return fail(QMC_EINVAL, "null plan_out");
  *plan_out = nullptr;
  std::unique_ptr<BatchPlan> bp(new BatchPlan());
  bp->src.assign(problems, problems + (problems && count > 0 ? count : 0));
  int rc = batch_create(bp.get(), count, problems, 1ull << 20);
  if (rc) {
    batch_release(bp.get());
    return rc;
  }
  *plan_out = reinterpret_cast<qmc_batch_plan>(bp.release());
  return QMC_OK;
}

int qmc_batch_plan_execute(qmc_batch_plan plan, qmc_result* out, double* per_shift, void* stream) {
  if (!plan) return fail(QMC_EINVAL, "null plan");
  return batch_execute(reinterpret_cast<BatchPlan*>(plan), out, per_shift, (cudaStream_t)stream);
}

int qmc_batch_plan_destroy(qmc_batch_plan plan) {
  if (!plan) return QMC_OK;
  BatchPlan* bp = reinterpret_cast<BatchPlan*>(plan);
  cudaDeviceSynchronize();
  batch_release(bp);
  delete bp;
  return QMC_OK;
}

int qmc_batch_plan_launches(qmc_batch_plan plan, int32_t* launches_out) {
  if (!plan || !launches_out) return fail(QMC_EINVAL, "null argument");
  *launches_out = reinterpret_cast<BatchPlan*>(plan)->launches;
  return QMC_OK;
}

int qmc_batch_plan_tune(qmc_batch_plan plan, const qmc_problem* problems, void* stream, uint64_t* work_per_cta_out) {
  if (!plan || !problems) return fail(QMC_EINVAL, "null argument");
  BatchPlan* bp = reinterpret_cast<BatchPlan*>(plan);
  cudaStream_t st = (cudaStream_t)stream;
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return fail(QMC_ECUDA, "events");
  std::vector<qmc_result> scratch(bp->count);
  float best_ms = 1e30f;
  uint64_t best_w = bp->work_per_cta;
  int rc = QMC_OK;
  for (int lw = 18; lw <= 24 && rc == QMC_OK; ++lw) {
    const uint64_t w = 1ull << lw;
    BatchPlan trial;
    rc = batch_create(&trial, bp->count, problems, w);
    if (rc) break;
    float tot = 0.0f;
    for (int rep = 0; rep < 4 && rc == QMC_OK; ++rep) {
      cudaEventRecord(a, st);
      if (cudaGraphLaunch(trial.exec, st) != cudaSuccess) rc = fail(QMC_ECUDA, "tuning launch");
      cudaEventRecord(b, st);
      cudaEventSynchronize(b);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, a, b);
      if (rep > 0) tot += ms;  // first replay warms up
    }
    cudaStreamSynchronize(st);
    batch_release(&trial);
    if (tot > 0.0f && tot < best_ms) {
      best_ms = tot;
      best_w = w;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  if (best_w != bp->work_per_cta) {
    cudaStreamSynchronize(st);
    batch_release(bp);
    rc = batch_create(bp, bp->count, problems, best_w);
    if (rc) return rc;
  }
  if (work_per_cta_out) *work_per_cta_out = best_w;
  return QMC_OK;
}

int qmc_integrate_batch(int32_t count, const qmc_problem* problems, qmc_result* out, double* per_shift,
                        void* stream) {
  BatchPlan bp;
  int rc = batch_create(&bp, count, problems, 1ull << 20);
  if (rc == QMC_OK) rc = batch_execute(&bp, out, per_shift, (cudaStream_t)stream);
  cudaStreamSynchronize((cudaStream_t)stream);
  batch_release(&bp);
  return rc;
}

}  // extern "C"

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
#include <cmath>
#include <cstdlib>
#include <string>
#include <thread>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
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
  // persistent mode: one launch over (descriptor, j-chunk) work items
  bool persistent = false;
  uint32_t chunk = 1u << 16;
  struct Sector {
    int m = 0;
    uint64_t n = 0;
    int nitems = 0;
    double final_scale = 1.0;
  };
  std::vector<Sector> psec;
  std::vector<int> pdesc_sector;         // descriptor -> sector
  std::vector<PersistDesc> pdesc;
  std::vector<PersistItem> pitems;
  PersistDesc* pdesc_dev = nullptr;
  PersistItem* pitems_dev = nullptr;
  unsigned* pnext_dev = nullptr;
  int pgrid = 0;
  int pmc = kPersistMc;                  // shift rows per descriptor
  void* pj_fn = nullptr;                 // run-time specialised persistent kernel (CUfunction), if any
  int pj_occ = 0;
  int pj_min_ctas = 1;                   // CTAs per SM it is built for (1, or 2 at 128 registers)
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

// ---------------------------------------------------------- persistent --

// Descriptors (one per sector and chunk of `mc` shifts: kPersistMc for the
// generic kernel, kPjMc for the specialised one) and the work list, longest
// items first.
static int persist_build(BatchPlan* bp, int32_t count, const qmc_problem* problems, uint32_t chunk, int mc) {
  if (count < 1 || count > 65536) return fail(QMC_EINVAL, "batch count=%d outside [1, 65536]", count);
  if (!problems) return fail(QMC_EINVAL, "null problems");
  if (chunk < (uint32_t)kThreads || chunk % kThreads != 0 || chunk > (1u << 24))
    return fail(QMC_EINVAL, "chunk of %u points: a multiple of %d in [%d, 2^24]", chunk, kThreads, kThreads);
  bp->count = count;
  bp->persistent = true;
  bp->chunk = chunk;
  bp->pmc = mc;
  bp->psec.assign(count, BatchPlan::Sector());
  bp->pdesc.clear();
  bp->pdesc_sector.clear();
  bp->pitems.clear();
  bp->ps_off.clear();
  bp->total_m = 0;
  bp->max_m = 0;
  struct Cost {
    double c;
    PersistItem it;
  };
  std::vector<Cost> costs;
  for (int s = 0; s < count; ++s) {
    const qmc_problem& q = problems[s];
    int rc = validate_problem(q.d, q.n, q.m, q.g, q.shifts, q.t, q.f);
    if (rc) {
      const std::string why = qmc_last_error();
      return fail(rc, "problem %d: %s", s, why.c_str());
    }
    const qmc_integrand& f = *q.f;
    const bool tr_ok = q.t.kind != QMC_TRANSFORM_KOROBOV || q.t.alpha == 3;
    if (f.kind != QMC_F_SECTOR || f.precision != QMC_FP32EVAL || f.aU != -2 || f.aF != -1 || q.d > kDFast ||
        poly_degree(f.U, q.d) > 1 || poly_degree(f.F, q.d) > 2 || !tr_ok)
      return fail(QMC_EUNSUPPORTED,
                  "problem %d: the persistent batch takes FP32EVAL U^-2 F^-1 sectors, deg U <= 1, deg F <= 2, "
                  "d <= %d, transform none, baker or Korobov 3", s, kDFast);
    RuleParams<float> base;
    fill_common(base, q.d, q.n, q.g, q.t, &f);
    auto cu = pack_dense(f.U, q.d, 1);
    auto cf = pack_dense(f.F, q.d, 2);
    prescale_slots(cu.data(), q.d, 1, fx_sigma(base.tr));
    prescale_slots(cf.data(), q.d, 2, fx_sigma(base.tr));
    for (size_t i = 0; i < cu.size(); ++i) base.cU[i] = (float)cu[i];
    for (size_t i = 0; i < cf.size(); ++i) base.cF[i] = (float)cf[i];
    fill_pairs(base, q.d);  // check_finite: set by fill_common (off when U, F > 0 on the cube)
    base.m_total = q.m;
    BatchPlan::Sector& sec = bp->psec[s];
    sec.m = q.m;
    sec.n = q.n;
    sec.nitems = (int)((q.n + chunk - 1) / chunk);
    sec.final_scale = base.tr == TR_KOROBOV ? std::pow((double)base.kor[7], (double)q.d) : 1.0;
    bp->ps_off.push_back((size_t)bp->total_m * 2);
    bp->total_m += q.m;
    bp->max_m = std::max(bp->max_m, q.m);
    const double per_point = (double)(poly_slots(q.d, 1) + poly_slots(q.d, 2) + 2 * q.d);
    for (int k0 = 0; k0 < q.m; k0 += mc) {
      const int mk = std::min(mc, q.m - k0);
      PersistDesc D;
      std::memset(&D, 0, sizeof(D));
      D.P = base;
      D.P.m_launch = mk;
      D.P.k_base = k0;
      for (int kk = 0; kk < mc; ++kk)  // rows mk.. repeat row k0 (evaluated, never written back)
        for (int i = 0; i < q.d; ++i)
          set_shift(D.P, kk, i, shift_fixed64(q.shifts[(size_t)(kk < mk ? k0 + kk : k0) * q.d + i]));
      D.nitems = sec.nitems;
      const uint32_t di = (uint32_t)bp->pdesc.size();
      bp->pdesc.push_back(D);
      bp->pdesc_sector.push_back(s);
      for (int it = 0; it < sec.nitems; ++it) {
        const uint64_t pts = std::min<uint64_t>(chunk, q.n - (uint64_t)it * chunk);
        costs.push_back({(double)pts * per_point * mc, PersistItem{di, (uint32_t)it}});
      }
    }
  }
  if (costs.size() > 0xFFFFFFF0ull) return fail(QMC_EINVAL, "too many work items (%zu)", costs.size());
  std::stable_sort(costs.begin(), costs.end(), [](const Cost& a, const Cost& b) { return a.c > b.c; });
  bp->pitems.reserve(costs.size());
  for (const Cost& c : costs) bp->pitems.push_back(c.it);
  bp->launches = 2;  // the persistent kernel and the final pass
  return QMC_OK;
}

static int persist_alloc(BatchPlan* bp) {
  size_t bytes = 0;
  std::vector<size_t> part_off(bp->count), cnt_off(bp->count);
  for (int i = 0; i < bp->count; ++i) {
    part_off[i] = bytes;
    bytes += (size_t)bp->psec[i].m * bp->psec[i].nitems * 2 * sizeof(double);
  }
  for (int i = 0; i < bp->count; ++i) {
    cnt_off[i] = bytes;
    bytes += 2 * sizeof(unsigned long long);
  }
  const size_t next_off = bytes;
  bytes += 16;
  bytes = (bytes + 255) & ~(size_t)255;
  const size_t res_off = bytes;
  bytes += (size_t)bp->count * sizeof(qmc_result);
  bytes = (bytes + 255) & ~(size_t)255;
  const size_t ps_off = bytes;
  bytes += (size_t)bp->total_m * 2 * sizeof(double);
  bytes = (bytes + 255) & ~(size_t)255;
  const size_t fin_off = bytes;
  bytes += (size_t)bp->count * sizeof(FinalizeArgs);
  bytes = (bytes + 255) & ~(size_t)255;
  const size_t desc_off = bytes;
  bytes += bp->pdesc.size() * sizeof(PersistDesc);
  bytes = (bytes + 255) & ~(size_t)255;
  const size_t item_off = bytes;
  bytes += bp->pitems.size() * sizeof(PersistItem);
  cudaError_t e = cudaMalloc(&bp->ws, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(QMC_ENOMEM, "persistent batch workspace of %zu bytes: %s", bytes, cudaGetErrorString(e));
  }
  char* base = (char*)bp->ws;
  bp->res_dev = (qmc_result*)(base + res_off);
  bp->ps_dev = (double*)(base + ps_off);
  bp->fin_dev = (FinalizeArgs*)(base + fin_off);
  bp->pdesc_dev = (PersistDesc*)(base + desc_off);
  bp->pitems_dev = (PersistItem*)(base + item_off);
  bp->pnext_dev = (unsigned*)(base + next_off);
  bp->fin_host.resize(bp->count);
  for (int i = 0; i < bp->count; ++i) {
    const BatchPlan::Sector& sec = bp->psec[i];
    FinalizeArgs& A = bp->fin_host[i];
    std::memset(&A, 0, sizeof(A));
    A.partial = (double*)(base + part_off[i]);
    A.nblk = sec.nitems;
    A.m = sec.m;
    A.is_complex = 0;
    A.dn = (double)sec.n;
    A.value_scale = sec.final_scale;
    A.counters = (unsigned long long*)(base + cnt_off[i]);
    A.result = bp->res_dev + i;
    A.per_shift = bp->ps_dev + bp->ps_off[i];
  }
  for (size_t q = 0; q < bp->pdesc.size(); ++q) {
    const int s = bp->pdesc_sector[q];
    bp->pdesc[q].partial = (double*)(base + part_off[s]);
    bp->pdesc[q].counters = (unsigned long long*)(base + cnt_off[s]);
  }
  e = cudaMemcpy(bp->fin_dev, bp->fin_host.data(), (size_t)bp->count * sizeof(FinalizeArgs), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(bp->pdesc_dev, bp->pdesc.data(), bp->pdesc.size() * sizeof(PersistDesc), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(bp->pitems_dev, bp->pitems.data(), bp->pitems.size() * sizeof(PersistItem), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(base + cnt_off[0], 0, (size_t)bp->count * 2 * sizeof(unsigned long long) + 16);
  if (e != cudaSuccess) return cuda_fail(e, "persistent batch descriptors");
  int occ = bp->pj_occ;
  if (!bp->pj_fn) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, persist_kernel_ptr(), kThreads, 0);
    if (e != cudaSuccess) return cuda_fail(e, "persistent kernel occupancy");
  }
  const int sms = device_sms();
  if (sms <= 0) return fail(QMC_ECUDA, "no CUDA device");
  bp->pgrid = (int)std::min<uint64_t>((uint64_t)sms * (uint64_t)std::max(occ, 1), bp->pitems.size());
  return QMC_OK;
}

// counter reset -> persistent kernel -> final pass
static int persist_graph(BatchPlan* bp) {
  cudaError_t e = cudaGraphCreate(&bp->graph, 0);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphCreate");
  cudaMemsetParams mp;
  std::memset(&mp, 0, sizeof(mp));
  mp.dst = bp->pnext_dev;
  mp.value = 0;
  mp.elementSize = 4;
  mp.width = 1;
  mp.height = 1;
  mp.pitch = 4;
  cudaGraphNode_t mnode;
  e = cudaGraphAddMemsetNode(&mnode, bp->graph, nullptr, 0, &mp);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphAddMemsetNode");
  PersistArgs A;
  std::memset(&A, 0, sizeof(A));
  A.descs = bp->pdesc_dev;
  A.items = bp->pitems_dev;
  A.nitems = (uint32_t)bp->pitems.size();
  A.chunk = bp->chunk;
  A.next = bp->pnext_dev;
  void* kargs[1] = {&A};
  cudaGraphNode_t knode;
  if (bp->pj_fn) {
    Launch ln;
    ln.cufunc = bp->pj_fn;
    ln.grid = dim3(bp->pgrid);
    int rc = graph_add_launch(bp->graph, ln, kargs, &knode, &mnode, 1);
    if (rc) return rc;
  } else {
    cudaKernelNodeParams kp;
    std::memset(&kp, 0, sizeof(kp));
    kp.func = (void*)persist_kernel_ptr();
    kp.gridDim = dim3(bp->pgrid);
    kp.blockDim = dim3(kThreads);
    kp.kernelParams = kargs;
    e = cudaGraphAddKernelNode(&knode, bp->graph, &mnode, 1, &kp);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphAddKernelNode (persistent kernel)");
  }
  FinalizeArgs* fin = bp->fin_dev;
  void* fargs[1] = {&fin};
  cudaKernelNodeParams fp;
  std::memset(&fp, 0, sizeof(fp));
  fp.func = (void*)finalize_batch_ptr();
  fp.gridDim = dim3(bp->count);
  fp.blockDim = dim3(256);
  fp.sharedMemBytes = (unsigned)((size_t)bp->max_m * 2 * sizeof(double));
  fp.kernelParams = fargs;
  cudaGraphNode_t fnode;
  e = cudaGraphAddKernelNode(&fnode, bp->graph, &knode, 1, &fp);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphAddKernelNode (final pass)");
  e = cudaGraphInstantiate(&bp->exec, bp->graph, 0);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  return QMC_OK;
}

// QMC_PERSIST_JIT=0 keeps persistent plans on the generic kernel.
static bool persist_jit_enabled() {
  const char* e = std::getenv("QMC_PERSIST_JIT");
  return jit_enabled() && !(e && e[0] == '0');
}

// The run-time specialisation's view of the descriptors persist_build made:
// one PjSector per problem (its lattice, dense slots, Korobov coefficients)
// and one PjDesc per descriptor (its shift rows).
static void persist_descriptors(const BatchPlan* bp, std::vector<PjSector>* secs_out, std::vector<PjDesc>* descs_out) {
  std::vector<PjSector>& secs = *secs_out;
  std::vector<PjDesc>& descs = *descs_out;
  secs.assign(bp->count, PjSector());
  descs.assign(bp->pdesc.size(), PjDesc());
  std::vector<bool> have(bp->count, false);
  for (size_t q = 0; q < bp->pdesc.size(); ++q) {
    const RuleParams<float>& P = bp->pdesc[q].P;
    const int s = bp->pdesc_sector[q];
    if (!have[s]) {
      PjSector& S = secs[s];
      S.d = P.d;
      S.tr = P.tr;
      S.check = P.check_finite != 0;
      S.n = P.n;
      S.rc = P.rc;
      for (int i = 0; i < P.d; ++i) {
        S.g[i] = P.g[i];
        S.gstep[i] = P.gstep[i];
      }
      S.cu.assign(P.cU, P.cU + poly_slots(P.d, 1));
      S.cf.assign(P.cF, P.cF + poly_slots(P.d, 2));
      for (int k = 0; k < 8; ++k) S.kor[k] = P.kor[k];
      have[s] = true;
    }
    PjDesc& Dq = descs[q];
    Dq.sector = s;
    Dq.kbase = P.k_base;
    Dq.m = P.m_launch;
    Dq.mc = std::min(kPjMc, (P.m_launch + 1) & ~1);
    Dq.shift.resize((size_t)Dq.mc * P.d);
    for (int k = 0; k < Dq.mc; ++k)
      for (int i = 0; i < P.d; ++i) Dq.shift[(size_t)k * P.d + i] = P.shiftx[k][i];
  }
  // every Korobov sector takes weight 3: its coefficients serve the whole module
  for (int s = 0; s < bp->count; ++s)
    if (secs[s].tr == TR_KOROBOV) {
      for (int t = 0; t < bp->count; ++t) std::memcpy(secs[t].kor, secs[s].kor, sizeof(secs[s].kor));
      break;
    }
}

// The specialised persistent kernel for the descriptors persist_build made
// (kPjMc shift rows each); false if it cannot be built (the caller falls back).
static bool persist_specialise(BatchPlan* bp) {
  std::vector<PjSector> secs;
  std::vector<PjDesc> descs;
  persist_descriptors(bp, &secs, &descs);
  void* fn = nullptr;
  int occ = 0;
  if (jit_persist(secs, descs, bp->pj_min_ctas, &fn, &occ) != QMC_OK) return false;
  bp->pj_fn = fn;
  bp->pj_occ = occ;
  return true;
}

static int persist_create(BatchPlan* bp, int32_t count, const qmc_problem* problems, uint32_t chunk,
                          int min_ctas = 1) {
  bp->pj_min_ctas = min_ctas;
  bp->pj_fn = nullptr;
  bp->pj_occ = 0;
  int rc = QMC_OK;
  bool specialised = false;
  if (persist_jit_enabled()) {
    rc = persist_build(bp, count, problems, chunk, kPjMc);
    if (rc) return rc;
    specialised = persist_specialise(bp);
  }
  if (!specialised) {
    rc = persist_build(bp, count, problems, chunk, kPersistMc);
    if (rc) return rc;
  }
  rc = persist_alloc(bp);
  if (rc) return rc;
  return persist_graph(bp);
}

static int batch_create(BatchPlan* bp, int32_t count, const qmc_problem* problems, uint64_t work_per_cta) {
  int rc = batch_build(bp, count, problems, work_per_cta);
  if (rc) return rc;
  rc = batch_alloc(bp);
  if (rc) return rc;
  return batch_graph(bp);
}

// Results and per-shift values of the last run into the caller's buffers
// (stream-ordered).
static int batch_copy_out(BatchPlan* bp, qmc_result* out, double* per_shift, cudaStream_t stream) {
  const bool out_dev = is_device_pointer(out);
  const bool ps_dev = per_shift ? is_device_pointer(per_shift) : true;
  cudaError_t e = cudaMemcpyAsync(out, bp->res_dev, (size_t)bp->count * sizeof(qmc_result),
                                  out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch results");
  if (per_shift) {
    e = cudaMemcpyAsync(per_shift, bp->ps_dev, (size_t)bp->total_m * 2 * sizeof(double),
                        ps_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, stream);
    if (e != cudaSuccess) return cuda_fail(e, "batch per-shift values");
  }
  return QMC_OK;
}

// ------------------------------------------------------------ one shot --
//
// qmc_integrate_batch runs a batch once.  Building and instantiating a CUDA
// graph, and cudaMalloc / cudaFree (which waits for the whole device), cost
// more host time than one run needs, and at the sizes of a tolerance walk's
// later levels more than the batch's device time.  The one-shot path takes
// its workspace from the stream-ordered pool (cudaMallocAsync and
// cudaFreeAsync on the caller's stream) and launches every problem's kernels
// directly, round-robin over kOneShotStreams internal streams forked from the
// caller's stream by an event and joined back before the final pass, so the
// sectors still run side by side.
constexpr int kOneShotStreams = 8;
// evaluations per CTA of a one-shot batch (a problem gets ceil(n m / W) CTAs,
// at most 4 per SM).  Sectors run side by side on 8 streams, so a pass of
// many medium sectors fills the GPU only if each gets enough CTAs: the C3
// walks to 1e-8 under Korobov 3 took 52 / 51 / 50 ms at W = 2^18 / 2^17 /
// 2^16 (49 / 44 / 42 ms when started at the ladder's bottom)
constexpr uint64_t kOneShotWork = 1ull << 16;
constexpr int kOneShotMaxDevices = 64;
struct OneShotStreams {
  cudaStream_t s[kOneShotStreams] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kOneShotStreams] = {};
  bool ok = false;
};
static std::mutex g_oneshot_mu;  // guards the streams' events between record and wait
static OneShotStreams g_oneshot[kOneShotMaxDevices];

static int oneshot_streams(OneShotStreams** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kOneShotMaxDevices) return fail(QMC_EUNSUPPORTED, "device index %d too large", dev);
  OneShotStreams& S = g_oneshot[dev];
  if (!S.ok) {
    e = cudaEventCreateWithFlags(&S.fork, cudaEventDisableTiming);
    for (int k = 0; k < kOneShotStreams && e == cudaSuccess; ++k) {
      e = cudaStreamCreateWithFlags(&S.s[k], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S.join[k], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return cuda_fail(e, "batch streams");
    S.ok = true;
  }
  *out = &S;
  return QMC_OK;
}

// Every launch of problems idx[0..nidx) (all problems when idx is null),
// round-robin over the internal streams forked from `stream` and joined back
// to it.
static int launch_side_by_side(BatchPlan* bp, const int* idx, int nidx, cudaStream_t stream) {
  OneShotStreams* S = nullptr;
  int rc = oneshot_streams(&S);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_oneshot_mu);
  cudaError_t e = cudaEventRecord(S->fork, stream);
  for (int k = 0; k < kOneShotStreams && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(S->s[k], S->fork, 0);
  if (e != cudaSuccess) return cuda_fail(e, "batch fork");
  SampleIO none;
  std::memset(&none, 0, sizeof(none));
  for (int u = 0; u < nidx && rc == QMC_OK; ++u) {
    Plan* pl = bp->probs[idx ? idx[u] : u].get();
    for (Launch& ln : pl->launches) {
      double* partial = pl->ws.partial;
      unsigned long long* counters = pl->ws.counters;
      void* args[4] = {(void*)ln.params.data(), &partial, &counters, &none};
      rc = launch_any(ln, ln.grid, args, S->s[u % kOneShotStreams]);
      if (rc) break;
    }
  }
  // join every internal stream back, even after a failed launch
  for (int k = 0; k < kOneShotStreams; ++k) {
    cudaEventRecord(S->join[k], S->s[k]);
    cudaStreamWaitEvent(stream, S->join[k], 0);
  }
  return rc;
}

static int oneshot_run(BatchPlan* bp, cudaStream_t stream) {
  size_t bytes = 0;
  std::vector<size_t> part_off(bp->count), cnt_off(bp->count);
  for (int i = 0; i < bp->count; ++i) {
    part_off[i] = bytes;
    bytes += (size_t)bp->probs[i]->m * bp->probs[i]->nblk * 2 * sizeof(double);
  }
  for (int i = 0; i < bp->count; ++i) {
    cnt_off[i] = bytes;
    bytes += 2 * sizeof(unsigned long long);
  }
  const size_t cnt_bytes = bytes - cnt_off[0];
  bytes = (bytes + 255) & ~(size_t)255;
  const size_t res_off = bytes;
  bytes += (size_t)bp->count * sizeof(qmc_result);
  bytes = (bytes + 255) & ~(size_t)255;
  const size_t ps_off = bytes;
  bytes += (size_t)bp->total_m * 2 * sizeof(double);
  bytes = (bytes + 255) & ~(size_t)255;
  const size_t fin_off = bytes;
  bytes += (size_t)bp->count * sizeof(FinalizeArgs);
  cudaError_t e = cudaMallocAsync(&bp->ws, bytes, stream);
  if (e != cudaSuccess) {
    bp->ws = nullptr;
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
  e = cudaMemcpyAsync(bp->fin_dev, bp->fin_host.data(), (size_t)bp->count * sizeof(FinalizeArgs),
                      cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + cnt_off[0], 0, cnt_bytes, stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch descriptors");
  int rc = launch_side_by_side(bp, nullptr, bp->count, stream);
  if (rc) return rc;
  FinalizeArgs* fin = bp->fin_dev;
  void* fargs[1] = {&fin};
  e = cudaLaunchKernel(finalize_batch_ptr(), dim3(bp->count), dim3(256), fargs, (size_t)bp->max_m * 2 * sizeof(double),
                       stream);
  if (e != cudaSuccess) return cuda_fail(e, "batch final pass");
  return QMC_OK;
}

// ------------------------------------------------------ ladder walk --
//
// qmc_integrate_batch_to_tolerance.  Every problem's plan (kernel, shifts,
// coefficients) is built once, on its own lattice; a later level only moves
// the plan to the next lattice (plan_rebase: n, g, the reciprocal of n and
// the launch shape), so a pass costs the launches of the problems that move
// up, one final pass over them and one copy of the results.

constexpr uint64_t kWalkWork = kOneShotWork;  // evaluations per CTA, as qmc_integrate_batch

static int walk_cap(uint64_t n, int m, int sms) {
  const uint64_t evals = n * (uint64_t)std::max(m, 1);
  return (int)std::max<uint64_t>(1, std::min<uint64_t>((evals + kWalkWork - 1) / kWalkWork, 4ull * sms));
}

// One pass: the listed problems' rules, their final pass, and every
// problem's current result copied to res (host), and with ps every
// problem's per-shift values ([total_m][2], host).
static int walk_pass(BatchPlan* bp, const std::vector<int>& act, std::vector<FinalizeArgs>& fin,
                     std::vector<qmc_result>& res, cudaStream_t stream, double* ps = nullptr) {
  fin.resize(act.size());
  for (size_t u = 0; u < act.size(); ++u) {
    const int i = act[u];
    const Plan* pl = bp->probs[i].get();
    FinalizeArgs& A = fin[u];
    std::memset(&A, 0, sizeof(A));
    A.partial = pl->ws.partial;
    A.nblk = pl->nblk;
    A.m = pl->m;
    A.is_complex = pl->is_complex;
    A.groups = 1;
    A.dn = (double)pl->n;
    A.value_scale = pl->final_scale;
    A.offset[0] = pl->offset[0];
    A.offset[1] = pl->offset[1];
    A.counters = pl->ws.counters;
    A.result = bp->res_dev + i;
    A.per_shift = bp->ps_dev + bp->ps_off[i];
  }
  cudaError_t e = cudaMemcpyAsync(bp->fin_dev, fin.data(), fin.size() * sizeof(FinalizeArgs), cudaMemcpyHostToDevice,
                                  stream);
  if (e != cudaSuccess) return cuda_fail(e, "walk descriptors");
  int rc = launch_side_by_side(bp, act.data(), (int)act.size(), stream);
  if (rc) return rc;
  FinalizeArgs* fd = bp->fin_dev;
  void* fargs[1] = {&fd};
  e = cudaLaunchKernel(finalize_batch_ptr(), dim3((unsigned)act.size()), dim3(256), fargs,
                       (size_t)bp->max_m * 2 * sizeof(double), stream);
  if (e != cudaSuccess) return cuda_fail(e, "walk final pass");
  e = cudaMemcpyAsync(res.data(), bp->res_dev, res.size() * sizeof(qmc_result), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess && ps)
    e = cudaMemcpyAsync(ps, bp->ps_dev, (size_t)bp->total_m * 2 * sizeof(double), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(e, "walk results");
  return QMC_OK;
}

// Persistent passes (QMC_WALK_PERSISTENT): every pass is one launch of the
// run-time specialised persistent kernel built with run-time lattices
// (qmc_jit_walk): each (sector, chunk of 16 shifts) keeps its compiled shifts
// and coefficients, and the pass hands each descriptor its sector's current
// lattice and slots.  Work items of kWalkChunk points from all refined
// sectors, the costliest sectors' first, feed one wave of CTAs, so small and
// large sectors share the GPU in a single launch.  The module is compiled for
// one CTA per SM (255 registers): with the lattice in registers (n, its
// reciprocal, g and gstep per dimension) it ran faster that way than at two CTAs
// per SM and 128 registers.
constexpr uint32_t kWalkChunk = 1u << 15;

struct WalkPersist {
  void* fn = nullptr;                       // qmc_jit_walk (CUfunction)
  int occ = 0;
  int sms = 0;
  std::vector<std::vector<int>> descs_of;   // sector -> its descriptors
  std::vector<int> desc_mc;                 // descriptor -> shift rows evaluated
  std::vector<double> weight;               // sector -> cost of a point per shift row
  std::vector<PjLattice> lat;               // descriptor -> lattice and slots (host copy)
  std::vector<double*> part;                // sector -> slots
  std::vector<unsigned long long*> cnt;     // sector -> counters
  std::vector<int> nitems;                  // sector -> items at its current lattice
  PjLattice* lat_dev = nullptr;
  PersistItem* items_dev = nullptr;
  unsigned* next_dev = nullptr;
};

// Descriptors, the run-time lattice module and the host tables; slots are
// placed by the caller.
static int walk_persist_build(BatchPlan* bp, WalkPersist* W, int32_t count, const qmc_problem* problems) {
  int rc = persist_build(bp, count, problems, kWalkChunk, kPjMc);
  if (rc) return rc;
  std::vector<PjSector> secs;
  std::vector<PjDesc> descs;
  persist_descriptors(bp, &secs, &descs);
  if (!jit_enabled()) return fail(QMC_EUNSUPPORTED, "persistent walk passes need run-time compilation (QMC_JIT)");
  rc = jit_persist(secs, descs, 1, &W->fn, &W->occ, true);
  if (rc) return fail(rc == QMC_EUNSUPPORTED ? QMC_EUNSUPPORTED : rc, "the persistent walk kernel could not be built");
  W->sms = device_sms();
  if (W->sms <= 0) return fail(QMC_ECUDA, "no CUDA device");
  W->descs_of.assign(count, std::vector<int>());
  W->desc_mc.resize(descs.size());
  for (size_t q = 0; q < descs.size(); ++q) {
    W->descs_of[descs[q].sector].push_back((int)q);
    W->desc_mc[q] = descs[q].mc;
  }
  W->weight.resize(count);
  for (int s = 0; s < count; ++s)
    W->weight[s] = (double)(poly_slots(problems[s].d, 1) + poly_slots(problems[s].d, 2) + 2 * problems[s].d);
  W->lat.assign(descs.size(), PjLattice());
  W->part.assign(count, nullptr);
  W->cnt.assign(count, nullptr);
  W->nitems.assign(count, 0);
  return QMC_OK;
}

// One persistent pass over the listed sectors, each on its lattice (n[i],
// g[i]); every problem's current result copied to res (host).
static int walk_pass_persistent(BatchPlan* bp, WalkPersist* W, const std::vector<int>& act,
                                const std::vector<uint64_t>& n, const std::vector<const uint64_t*>& g,
                                const qmc_problem* problems, std::vector<FinalizeArgs>& fin,
                                std::vector<qmc_result>& res, cudaStream_t stream) {
  // work items, the costliest sectors' first (a point's cost times the shift
  // rows): every item but a sector's last has kWalkChunk points
  std::vector<int> order(act);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return W->weight[a] > W->weight[b]; });
  std::vector<PersistItem> items;
  for (int i : order) {
    const uint64_t ni = n[i];
    const int d = problems[i].d;
    const Recip rc = reciprocal(ni);
    W->nitems[i] = (int)((ni + kWalkChunk - 1) / kWalkChunk);
    for (int q : W->descs_of[i]) {
      PjLattice& L = W->lat[q];
      std::memset(&L, 0, sizeof(L));
      L.n = ni;
      L.rhi = rc.rhi;
      L.rlo = rc.rlo;
      for (int dd = 0; dd < d; ++dd) {
        L.g[dd] = (uint32_t)g[i][dd];
        L.gstep[dd] = (uint32_t)(((uint64_t)kThreads * g[i][dd]) % ni);
      }
      L.partial = W->part[i];
      L.counters = W->cnt[i];
      L.nitems = W->nitems[i];
      for (int it = 0; it < W->nitems[i]; ++it) items.push_back(PersistItem{(uint32_t)q, (uint32_t)it});
    }
  }
  fin.resize(act.size());
  for (size_t u = 0; u < act.size(); ++u) {
    const int i = act[u];
    FinalizeArgs& A = fin[u];
    std::memset(&A, 0, sizeof(A));
    A.partial = W->part[i];
    A.nblk = W->nitems[i];
    A.m = problems[i].m;
    A.groups = 1;
    A.dn = (double)n[i];
    A.value_scale = bp->psec[i].final_scale;
    A.counters = W->cnt[i];
    A.result = bp->res_dev + i;
    A.per_shift = bp->ps_dev + bp->ps_off[i];
  }
  cudaError_t e = cudaMemcpyAsync(W->lat_dev, W->lat.data(), W->lat.size() * sizeof(PjLattice), cudaMemcpyHostToDevice,
                                  stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(W->items_dev, items.data(), items.size() * sizeof(PersistItem), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bp->fin_dev, fin.data(), fin.size() * sizeof(FinalizeArgs), cudaMemcpyHostToDevice, stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(W->next_dev, 0, sizeof(unsigned), stream);
  if (e != cudaSuccess) return cuda_fail(e, "walk pass tables");
  PersistArgs A;
  std::memset(&A, 0, sizeof(A));
  A.items = W->items_dev;
  A.nitems = (uint32_t)items.size();
  A.chunk = kWalkChunk;
  A.next = W->next_dev;
  A.lats = W->lat_dev;
  Launch ln;
  ln.cufunc = W->fn;
  const uint64_t wave = (uint64_t)W->sms * (uint64_t)std::max(W->occ, 1);
  ln.grid = dim3((unsigned)std::max<uint64_t>(1, std::min<uint64_t>(wave, items.size())));
  void* args[1] = {&A};
  int rc = launch_any(ln, ln.grid, args, stream);
  if (rc) return rc;
  FinalizeArgs* fd = bp->fin_dev;
  void* fargs[1] = {&fd};
  e = cudaLaunchKernel(finalize_batch_ptr(), dim3((unsigned)act.size()), dim3(256), fargs,
                       (size_t)bp->max_m * 2 * sizeof(double), stream);
  if (e != cudaSuccess) return cuda_fail(e, "walk final pass");
  e = cudaMemcpyAsync(res.data(), bp->res_dev, res.size() * sizeof(qmc_result), cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(e, "walk results");
  return QMC_OK;
}

// QMC_WALK_JUMP.  A problem whose error err exceeds its target t (its share
// rel_tol |sum| / sqrt(count) of the sum's tolerance, or rel_tol |Qbar_i|)
// moves up to the first size n' with (n'/n)^6 >= err / t: as far as an
// error falling like n^-6 would need to reach the target.  The rates the
// paper reports for its integrals lie between n^-1 and n^-4, so for such
// problems the jump does not pass the size they need, and it skips the
// passes in between; error estimates that fall faster can be taken past
// it.  Without a target (|Qbar| = 0) the problem moves one step.
static void walk_targets(const std::vector<qmc_result>& r, int criterion, double rel_tol, std::vector<double>& t) {
  const size_t count = r.size();
  t.resize(count);
  if (criterion == QMC_WALK_SUM) {
    double sre = 0.0, sim = 0.0;
    for (size_t i = 0; i < count; ++i) {
      sre += r[i].mean[0];
      sim += r[i].mean[1];
    }
    const double share = rel_tol * std::hypot(sre, sim) / std::sqrt((double)count);
    for (size_t i = 0; i < count; ++i) t[i] = share;
  } else {
    for (size_t i = 0; i < count; ++i) t[i] = rel_tol * std::hypot(r[i].mean[0], r[i].mean[1]);
  }
}

// err / target, 1 (one step) without a target
static double walk_excess(const qmc_result& r, double target) {
  return target > 0.0 ? std::hypot(r.err[0], r.err[1]) / target : 1.0;
}

// the rate bound of the jumps: errors assumed to fall no faster than n^-kJumpPow
constexpr int kJumpPow = 6;

// whether a size ratio q = n'/n is still short of an excess e: q^kJumpPow < e
static bool jump_short(double q, double e) {
  double p = 1.0;
  for (int t = 0; t < kJumpPow; ++t) p *= q;
  return p < e;
}

static int batch_walk(int32_t count, const qmc_problem* problems, int32_t levels, const uint64_t* ladder_n,
                      const uint64_t* ladder_g, int32_t ladder_dim, double rel_tol, int32_t criterion,
                      qmc_result* out, int32_t* level_out, int32_t* passes_out, cudaStream_t stream) {
  if (count < 1 || count > 65536) return fail(QMC_EINVAL, "batch count=%d outside [1, 65536]", count);
  if (!problems || !out) return fail(QMC_EINVAL, "null problems or results");
  if (levels < 0 || levels > 64 || (levels > 0 && (!ladder_n || !ladder_g)))
    return fail(QMC_EINVAL, "ladder of %d lattices (0..64, with n and g)", levels);
  if (ladder_dim < 1 || ladder_dim > QMC_DMAX) return fail(QMC_EINVAL, "ladder_dim=%d outside [1, %d]", ladder_dim, QMC_DMAX);
  if (!(rel_tol > 0.0)) return fail(QMC_EINVAL, "rel_tol must be > 0");
  const bool pers = (criterion & QMC_WALK_PERSISTENT) != 0;
  const bool jump = (criterion & QMC_WALK_JUMP) != 0;
  criterion &= ~(QMC_WALK_PERSISTENT | QMC_WALK_JUMP);
  if (criterion != QMC_WALK_SUM && criterion != QMC_WALK_EACH) return fail(QMC_EINVAL, "unknown criterion %d", criterion);
  for (int l = 0; l < levels; ++l) {
    const uint64_t n = ladder_n[l];
    if (n < 2 || n >= (1ull << 31) || (l > 0 && n <= ladder_n[l - 1]))
      return fail(QMC_EINVAL, "ladder n[%d]=%llu: sizes must increase within [2, 2^31)", l, (unsigned long long)n);
    for (int i = 0; i < ladder_dim; ++i) {
      const uint64_t gi = ladder_g[(size_t)l * ladder_dim + i];
      if (gi < 1 || gi >= n) return fail(QMC_EINVAL, "ladder g[%d][%d]=%llu outside [1, n)", l, i, (unsigned long long)gi);
    }
  }
  for (int i = 0; i < count && levels > 0; ++i)
    if (problems[i].d > ladder_dim) return fail(QMC_EINVAL, "problem %d: d=%d above ladder_dim", i, problems[i].d);
  if (is_device_pointer(out)) return fail(QMC_EINVAL, "the results must be host memory");
  const int sms = device_sms();
  if (sms <= 0) return fail(QMC_ECUDA, "no CUDA device");
  BatchPlan bp;
  WalkPersist W;
  int rc = pers ? walk_persist_build(&bp, &W, count, problems) : batch_build(&bp, count, problems, kWalkWork);
  if (rc) return rc;
  // lattices of problem i: its own, then the ladder's entries above its n
  std::vector<int> next(count), at(count, -1);
  std::vector<uint64_t> cur_n(count);
  std::vector<const uint64_t*> cur_g(count);
  for (int i = 0; i < count; ++i) {
    int l = 0;
    while (l < levels && ladder_n[l] <= problems[i].n) ++l;
    next[i] = l;
    cur_n[i] = problems[i].n;
    cur_g[i] = problems[i].g;
  }
  // slots: the sector kernels' CTAs (at most one resident wave, and at most
  // the cap of the largest lattice), or the persistent passes' work items
  size_t bytes = 0;
  std::vector<size_t> part_off(count), cnt_off(count);
  size_t max_items = 0;
  for (int i = 0; i < count; ++i) {
    const uint64_t n_max = next[i] < levels ? ladder_n[levels - 1] : problems[i].n;
    int slots = 0;
    if (pers) {
      slots = (int)((n_max + kWalkChunk - 1) / kWalkChunk);
      max_items += (size_t)slots * W.descs_of[i].size();
    } else {
      const Plan* pl = bp.probs[i].get();
      slots = pl->nblk;
      if (next[i] < levels) {
        const int wave = sms * std::max(pl->grid_occ, 1);
        slots = std::max(slots, pl->grid_capped ? std::min(wave, walk_cap(n_max, pl->m, sms)) : wave);
      }
    }
    part_off[i] = bytes;
    bytes += (size_t)problems[i].m * slots * 2 * sizeof(double);
  }
  for (int i = 0; i < count; ++i) {
    cnt_off[i] = bytes;
    bytes += 2 * sizeof(unsigned long long);
  }
  const size_t cnt_bytes = bytes - cnt_off[0];
  bytes = (bytes + 255) & ~(size_t)255;
  const size_t res_off = bytes;
  bytes += (size_t)count * sizeof(qmc_result);
  bytes = (bytes + 255) & ~(size_t)255;
  const size_t ps_off = bytes;
  bytes += (size_t)bp.total_m * 2 * sizeof(double);
  bytes = (bytes + 255) & ~(size_t)255;
  const size_t fin_off = bytes;
  bytes += (size_t)count * sizeof(FinalizeArgs);
  size_t lat_off = 0, items_off = 0, next_off = 0;
  if (pers) {
    bytes = (bytes + 255) & ~(size_t)255;
    lat_off = bytes;
    bytes += W.lat.size() * sizeof(PjLattice);
    bytes = (bytes + 255) & ~(size_t)255;
    items_off = bytes;
    bytes += std::max<size_t>(max_items, 1) * sizeof(PersistItem);
    bytes = (bytes + 255) & ~(size_t)255;
    next_off = bytes;
    bytes += 16;
  }
  cudaError_t e = cudaMallocAsync(&bp.ws, bytes, stream);
  if (e != cudaSuccess) {
    bp.ws = nullptr;
    cudaGetLastError();
    return fail(QMC_ENOMEM, "walk workspace of %zu bytes: %s", bytes, cudaGetErrorString(e));
  }
  char* base = (char*)bp.ws;
  bp.res_dev = (qmc_result*)(base + res_off);
  bp.ps_dev = (double*)(base + ps_off);
  bp.fin_dev = (FinalizeArgs*)(base + fin_off);
  for (int i = 0; i < count; ++i) {
    if (pers) {
      W.part[i] = (double*)(base + part_off[i]);
      W.cnt[i] = (unsigned long long*)(base + cnt_off[i]);
    } else {
      bp.probs[i]->ws.partial = (double*)(base + part_off[i]);
      bp.probs[i]->ws.counters = (unsigned long long*)(base + cnt_off[i]);
    }
  }
  if (pers) {
    W.lat_dev = (PjLattice*)(base + lat_off);
    W.items_dev = (PersistItem*)(base + items_off);
    W.next_dev = (unsigned*)(base + next_off);
  }
  e = cudaMemsetAsync(base + cnt_off[0], 0, cnt_bytes, stream);  // the final pass resets them after each read
  if (e != cudaSuccess) rc = cuda_fail(e, "walk counters");
  std::vector<int> act(count);
  for (int i = 0; i < count; ++i) act[i] = i;
  std::vector<FinalizeArgs> fin;
  std::vector<qmc_result> res(count);
  int passes = 0;
  bool reached = false;
  while (rc == QMC_OK) {
    if (passes > 0)
      for (int i : act) {
        const int l = next[i];
        cur_n[i] = ladder_n[l];
        cur_g[i] = ladder_g + (size_t)l * ladder_dim;
        if (!pers) {
          Plan* pl = bp.probs[i].get();
          rc = plan_rebase(pl, cur_n[i], cur_g[i], walk_cap(cur_n[i], pl->m, sms));
          if (rc) break;
        }
        at[i] = l;
        next[i] = l + 1;
      }
    if (rc) break;
    rc = pers ? walk_pass_persistent(&bp, &W, act, cur_n, cur_g, problems, fin, res, stream)
              : walk_pass(&bp, act, fin, res, stream);
    if (rc) break;
    ++passes;
    for (int i : act)
      if (res[i].status != QMC_OK && res[i].status != QMC_ENONFINITE && res[i].status != QMC_EDEFORM) {
        rc = fail(res[i].status, "problem %d failed with status %d", i, res[i].status);
        break;
      }
    if (rc) break;
    // next pass: the problems whose error is above their share of the tolerance
    act.clear();
    if (criterion == QMC_WALK_SUM) {
      double sre = 0.0, sim = 0.0, e2 = 0.0;
      for (int i = 0; i < count; ++i) {
        sre += res[i].mean[0];
        sim += res[i].mean[1];
        e2 += res[i].err[0] * res[i].err[0] + res[i].err[1] * res[i].err[1];
      }
      const double mag = std::hypot(sre, sim);
      if (mag > 0.0 && std::sqrt(e2) <= rel_tol * mag) {
        reached = true;
        break;
      }
      const double share = rel_tol * mag / std::sqrt((double)count);
      for (int i = 0; i < count; ++i)
        if (std::hypot(res[i].err[0], res[i].err[1]) > share && next[i] < levels) act.push_back(i);
    } else {
      bool all = true;
      for (int i = 0; i < count; ++i) {
        const double mag = std::hypot(res[i].mean[0], res[i].mean[1]);
        if (mag > 0.0 && std::hypot(res[i].err[0], res[i].err[1]) <= rel_tol * mag) continue;
        all = false;
        if (next[i] < levels) act.push_back(i);
      }
      if (all) {
        reached = true;
        break;
      }
    }
    if (act.empty()) break;
    if (jump) {
      std::vector<double> tgt;
      walk_targets(res, criterion, rel_tol, tgt);
      for (int i : act) {
        const double ex = walk_excess(res[i], tgt[i]);
        int l = next[i];
        while (l + 1 < levels && jump_short((double)ladder_n[l] / (double)cur_n[i], ex)) ++l;
        next[i] = l;
      }
    }
  }
  if (bp.ws) {
    cudaFreeAsync(bp.ws, stream);
    bp.ws = nullptr;
  }
  e = cudaStreamSynchronize(stream);
  if (rc == QMC_OK && e != cudaSuccess) rc = cuda_fail(e, "walk synchronise");
  if (rc) return rc;
  for (int i = 0; i < count; ++i) {
    out[i] = res[i];
    if (level_out) level_out[i] = at[i];
  }
  if (passes_out) *passes_out = passes;
  if (reached) return QMC_OK;
  if (criterion == QMC_WALK_EACH)
    for (int i = 0; i < count; ++i) {
      const double mag = std::hypot(out[i].mean[0], out[i].mean[1]);
      if (!(mag > 0.0 && std::hypot(out[i].err[0], out[i].err[1]) <= rel_tol * mag)) out[i].status = QMC_ETIMEOUT;
    }
  return fail(QMC_ETIMEOUT, "relative error %.3g not reached after %d passes", rel_tol, passes);
}

// ------------------------------------------------ embedded doubling walk --
//
// qmc_integrate_batch_extensible.  Problem i starts with the rule of n_i = 2^k
// points on the embedded vector g (g mod n_i).  A later pass doubles n_i and
// evaluates only the new points: they are the size-n_i lattice shifted by
// (g mod 2n_i) / (2n_i), so the plan moves to that lattice (plan_rebase) and
// takes the shifted shifts (plan_reshift).  The new per-shift values are
// averaged with the previous ones on the host, so every estimate is exactly
// the rule of its size and no point is evaluated twice.

static int batch_extensible(int32_t count, const qmc_problem* problems, int32_t levels, const uint64_t* g,
                            int32_t g_dim, double rel_tol, int32_t criterion, qmc_result* out, int32_t* level_out,
                            int32_t* passes_out, cudaStream_t stream) {
  if (count < 1 || count > 65536) return fail(QMC_EINVAL, "batch count=%d outside [1, 65536]", count);
  if (!problems || !out || !g) return fail(QMC_EINVAL, "null problems, generating vector or results");
  if (levels < 0 || levels > 30) return fail(QMC_EINVAL, "levels=%d outside [0, 30]", levels);
  if (g_dim < 1 || g_dim > QMC_DMAX) return fail(QMC_EINVAL, "g_dim=%d outside [1, %d]", g_dim, QMC_DMAX);
  if (!(rel_tol > 0.0)) return fail(QMC_EINVAL, "rel_tol must be > 0");
  const bool jump = (criterion & QMC_WALK_JUMP) != 0;
  criterion &= ~QMC_WALK_JUMP;
  if (criterion != QMC_WALK_SUM && criterion != QMC_WALK_EACH) return fail(QMC_EINVAL, "unknown criterion %d", criterion);
  for (int c = 0; c < g_dim; ++c)
    if ((g[c] & 1) == 0) return fail(QMC_EINVAL, "g[%d]=%llu must be odd", c, (unsigned long long)g[c]);
  std::vector<int> maxd(count);  // doublings each problem may take
  for (int i = 0; i < count; ++i) {
    const qmc_problem& q = problems[i];
    if (q.d < 1 || q.d > g_dim) return fail(QMC_EINVAL, "problem %d: d=%d outside [1, g_dim]", i, q.d);
    if (q.n < 2 || q.n > (1ull << 30) || (q.n & (q.n - 1)) != 0)
      return fail(QMC_EINVAL, "problem %d: n=%llu is not a power of two in [2, 2^30]", i, (unsigned long long)q.n);
    if (q.m < 2 || !q.shifts) return fail(QMC_EINVAL, "problem %d: m=%d shifts (the estimate needs m >= 2)", i, q.m);
    int k = 0;
    while ((1ull << k) < q.n) ++k;
    maxd[i] = std::min(levels, 30 - k);
  }
  if (is_device_pointer(out)) return fail(QMC_EINVAL, "the results must be host memory");
  const int sms = device_sms();
  if (sms <= 0) return fail(QMC_ECUDA, "no CUDA device");
  // the problems at their first size
  std::vector<qmc_problem> pr(problems, problems + count);
  std::vector<uint64_t> gm((size_t)count * g_dim);
  for (int i = 0; i < count; ++i) {
    for (int c = 0; c < pr[i].d; ++c) gm[(size_t)i * g_dim + c] = g[c] % pr[i].n;  // odd, so >= 1
    pr[i].g = gm.data() + (size_t)i * g_dim;
  }
  BatchPlan bp;
  int rc = batch_build(&bp, count, pr.data(), kWalkWork);
  if (rc) return rc;
  // slots: one resident wave, at most the cap of the largest rule evaluated
  // (half the last size; with jumps the last size itself)
  size_t bytes = 0;
  std::vector<size_t> part_off(count), cnt_off(count);
  for (int i = 0; i < count; ++i) {
    const Plan* pl = bp.probs[i].get();
    int slots = pl->nblk;
    if (maxd[i] > 0) {
      const uint64_t n_max = pr[i].n << (jump ? maxd[i] : maxd[i] - 1);
      const int wave = sms * std::max(pl->grid_occ, 1);
      slots = std::max(slots, pl->grid_capped ? std::min(wave, walk_cap(n_max, pl->m, sms)) : wave);
    }
    part_off[i] = bytes;
    bytes += (size_t)pl->m * slots * 2 * sizeof(double);
  }
  for (int i = 0; i < count; ++i) {
    cnt_off[i] = bytes;
    bytes += 2 * sizeof(unsigned long long);
  }
  const size_t cnt_bytes = bytes - cnt_off[0];
  bytes = (bytes + 255) & ~(size_t)255;
  const size_t res_off = bytes;
  bytes += (size_t)count * sizeof(qmc_result);
  bytes = (bytes + 255) & ~(size_t)255;
  const size_t ps_off = bytes;
  bytes += (size_t)bp.total_m * 2 * sizeof(double);
  bytes = (bytes + 255) & ~(size_t)255;
  const size_t fin_off = bytes;
  bytes += (size_t)count * sizeof(FinalizeArgs);
  cudaError_t e = cudaMallocAsync(&bp.ws, bytes, stream);
  if (e != cudaSuccess) {
    bp.ws = nullptr;
    cudaGetLastError();
    return fail(QMC_ENOMEM, "walk workspace of %zu bytes: %s", bytes, cudaGetErrorString(e));
  }
  char* base = (char*)bp.ws;
  bp.res_dev = (qmc_result*)(base + res_off);
  bp.ps_dev = (double*)(base + ps_off);
  bp.fin_dev = (FinalizeArgs*)(base + fin_off);
  for (int i = 0; i < count; ++i) {
    bp.probs[i]->ws.partial = (double*)(base + part_off[i]);
    bp.probs[i]->ws.counters = (unsigned long long*)(base + cnt_off[i]);
  }
  e = cudaMemsetAsync(base + cnt_off[0], 0, cnt_bytes, stream);  // the final pass resets them after each read
  if (e != cudaSuccess) rc = cuda_fail(e, "walk counters");
  const size_t tm2 = (size_t)bp.total_m * 2;
  std::vector<double> q(tm2), ps(tm2), sh;
  std::vector<uint64_t> size(count), gl(QMC_DMAX);
  std::vector<int> dbl(count, 0), step(count, 1);  // step: doublings of the next pass
  std::vector<unsigned long long> nonfinite(count, 0), deform(count, 0);
  std::vector<qmc_result> res(count), est(count);
  std::vector<FinalizeArgs> fin;
  std::vector<int> act(count);
  for (int i = 0; i < count; ++i) {
    act[i] = i;
    size[i] = pr[i].n;
  }
  int passes = 0;
  bool reached = false;
  while (rc == QMC_OK) {
    if (passes > 0)
      for (int i : act) {
        const qmc_problem& qp = problems[i];
        Plan* pl = bp.probs[i].get();
        if (step[i] > 1) {
          // a jump of several doublings: the whole rule of the new size
          const uint64_t n = size[i] << step[i];
          for (int c = 0; c < qp.d; ++c) gl[c] = g[c] % n;
          rc = plan_rebase(pl, n, gl.data(), walk_cap(n, pl->m, sms));
          if (rc == QMC_OK) rc = plan_reshift(pl, qp.shifts);
          if (rc) break;
          continue;
        }
        // the new points of size 2n: the size-n rule on shifts Delta + (g mod 2n) / (2n)
        const uint64_t n = size[i];
        for (int c = 0; c < qp.d; ++c) gl[c] = g[c] % n;
        rc = plan_rebase(pl, n, gl.data(), walk_cap(n, pl->m, sms));
        if (rc) break;
        sh.resize((size_t)qp.m * qp.d);
        const double two_n = (double)(2 * n);
        for (int k = 0; k < qp.m; ++k)
          for (int c = 0; c < qp.d; ++c) {
            const double v = qp.shifts[(size_t)k * qp.d + c] + (double)(g[c] % (2 * n)) / two_n;
            sh[(size_t)k * qp.d + c] = v >= 1.0 ? v - 1.0 : v;
          }
        rc = plan_reshift(pl, sh.data());
        if (rc) break;
      }
    if (rc) break;
    rc = walk_pass(&bp, act, fin, res, stream, ps.data());
    if (rc) break;
    for (int i : act) {
      if (res[i].status != QMC_OK && res[i].status != QMC_ENONFINITE && res[i].status != QMC_EDEFORM) {
        rc = fail(res[i].status, "problem %d failed with status %d", i, res[i].status);
        break;
      }
      double* qi = q.data() + bp.ps_off[i];
      const double* pi = ps.data() + bp.ps_off[i];
      const size_t m2 = (size_t)problems[i].m * 2;
      if (passes == 0) {
        std::memcpy(qi, pi, m2 * sizeof(double));
      } else if (step[i] > 1) {
        std::memcpy(qi, pi, m2 * sizeof(double));
        size[i] <<= step[i];
        dbl[i] += step[i];
      } else {
        for (size_t u = 0; u < m2; ++u) qi[u] = 0.5 * (qi[u] + pi[u]);
        size[i] *= 2;
        ++dbl[i];
      }
      nonfinite[i] += res[i].nonfinite;
      deform[i] += res[i].deform_violations;
      rc = qmc_combine_shifts(problems[i].m, qi, &est[i]);  // Eq. (3) on the size-size[i] rule's per-shift values
      if (rc) break;
      est[i].nonfinite = nonfinite[i];
      est[i].deform_violations = deform[i];
      est[i].status = nonfinite[i] ? QMC_ENONFINITE : (deform[i] ? QMC_EDEFORM : QMC_OK);
    }
    if (rc) break;
    ++passes;
    // next pass: the problems whose error is above their share of the tolerance
    act.clear();
    if (criterion == QMC_WALK_SUM) {
      double sre = 0.0, sim = 0.0, e2 = 0.0;
      for (int i = 0; i < count; ++i) {
        sre += est[i].mean[0];
        sim += est[i].mean[1];
        e2 += est[i].err[0] * est[i].err[0] + est[i].err[1] * est[i].err[1];
      }
      const double mag = std::hypot(sre, sim);
      if (mag > 0.0 && std::sqrt(e2) <= rel_tol * mag) {
        reached = true;
        break;
      }
      const double share = rel_tol * mag / std::sqrt((double)count);
      for (int i = 0; i < count; ++i)
        if (std::hypot(est[i].err[0], est[i].err[1]) > share && dbl[i] < maxd[i]) act.push_back(i);
    } else {
      bool all = true;
      for (int i = 0; i < count; ++i) {
        const double mag = std::hypot(est[i].mean[0], est[i].mean[1]);
        if (mag > 0.0 && std::hypot(est[i].err[0], est[i].err[1]) <= rel_tol * mag) continue;
        all = false;
        if (dbl[i] < maxd[i]) act.push_back(i);
      }
      if (all) {
        reached = true;
        break;
      }
    }
    if (act.empty()) break;
    if (jump) {
      std::vector<double> tgt;
      walk_targets(est, criterion, rel_tol, tgt);
      for (int i : act) {
        const double ex = walk_excess(est[i], tgt[i]);
        int k = 1;
        while (k < maxd[i] - dbl[i] && jump_short((double)(1ull << k), ex)) ++k;
        step[i] = k;
      }
    }
  }
  if (bp.ws) {
    cudaFreeAsync(bp.ws, stream);
    bp.ws = nullptr;
  }
  e = cudaStreamSynchronize(stream);
  if (rc == QMC_OK && e != cudaSuccess) rc = cuda_fail(e, "walk synchronise");
  if (rc) return rc;
  for (int i = 0; i < count; ++i) {
    out[i] = est[i];
    if (level_out) level_out[i] = dbl[i];
  }
  if (passes_out) *passes_out = passes;
  if (reached) return QMC_OK;
  if (criterion == QMC_WALK_EACH)
    for (int i = 0; i < count; ++i) {
      const double mag = std::hypot(out[i].mean[0], out[i].mean[1]);
      if (!(mag > 0.0 && std::hypot(out[i].err[0], out[i].err[1]) <= rel_tol * mag)) out[i].status = QMC_ETIMEOUT;
    }
  return fail(QMC_ETIMEOUT, "relative error %.3g not reached after %d passes", rel_tol, passes);
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

int qmc_batch_plan_create_persistent(int32_t count, const qmc_problem* problems, uint32_t chunk_points,
                                     qmc_batch_plan* plan_out) {
  if (!plan_out) return fail(QMC_EINVAL, "null plan_out");
  *plan_out = nullptr;
  std::unique_ptr<BatchPlan> bp(new BatchPlan());
  bp->src.assign(problems, problems + (problems && count > 0 ? count : 0));
  int rc = persist_create(bp.get(), count, problems, chunk_points ? chunk_points : (1u << 16));
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

int qmc_batch_plan_describe(qmc_batch_plan plan, char* buf, int32_t len) {
  if (!plan || !buf || len < 1) return fail(QMC_EINVAL, "null plan or buffer");
  const BatchPlan* bp = reinterpret_cast<const BatchPlan*>(plan);
  if (bp->persistent)
    snprintf(buf, (size_t)len, "mode=persistent specialised=%d problems=%d descriptors=%zu items=%zu ctas=%d chunk=%u "
             "shifts_per_descriptor=%d min_ctas=%d", bp->pj_fn ? 1 : 0, bp->count, bp->pdesc.size(), bp->pitems.size(),
             bp->pgrid, bp->chunk, bp->pmc, bp->pj_fn ? bp->pj_min_ctas : 0);
  else
    snprintf(buf, (size_t)len, "mode=graph problems=%d launches=%d work_per_cta=%llu", bp->count, bp->launches,
             (unsigned long long)bp->work_per_cta);
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
  float best_ms = 1e30f;
  const bool pers = bp->persistent;
  uint64_t best_w = pers ? bp->chunk : bp->work_per_cta;
  int best_minc = bp->pj_min_ctas;
  // a specialised persistent kernel is also built for two CTAs per SM (128 registers)
  const int max_minc = pers && bp->pj_fn ? 2 : 1;
  int rc = QMC_OK;
  const char* ve = std::getenv("QMC_TUNE_VERBOSE");  // per-candidate times on stderr
  const bool verbose = ve && ve[0] == '1';
  // graph mode: evaluations per CTA 2^18..2^24; persistent mode: points per work item 2^14..2^18
  for (int minc = 1; minc <= max_minc && rc == QMC_OK; ++minc)
    for (int lw = pers ? 14 : 18; lw <= (pers ? 18 : 24) && rc == QMC_OK; ++lw) {
      const uint64_t w = 1ull << lw;
      BatchPlan trial;
      rc = pers ? persist_create(&trial, bp->count, problems, (uint32_t)w, minc)
                : batch_create(&trial, bp->count, problems, w);
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
      const bool got = !pers || minc == 1 || trial.pj_fn;  // a failed two-CTA build fell back: not a candidate
      if (verbose)
        std::fprintf(stderr, "batch tune: %s work=2^%d min_ctas=%d%s ms=%.4f (mean of 3 replays)\n",
                     pers ? "persistent" : "graph", lw, pers ? minc : 0, got ? "" : " (not built)", tot / 3.0f);
      batch_release(&trial);
      if (got && tot > 0.0f && tot < best_ms) {
        best_ms = tot;
        best_w = w;
        best_minc = minc;
      }
    }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (rc) return rc;
  if (best_w != (pers ? (uint64_t)bp->chunk : bp->work_per_cta) || (pers && best_minc != bp->pj_min_ctas)) {
    cudaStreamSynchronize(st);
    batch_release(bp);
    rc = pers ? persist_create(bp, bp->count, problems, (uint32_t)best_w, best_minc)
              : batch_create(bp, bp->count, problems, best_w);
    if (rc) return rc;
  }
  if (work_per_cta_out) *work_per_cta_out = best_w;
  return QMC_OK;
}

int qmc_integrate_batch(int32_t count, const qmc_problem* problems, qmc_result* out, double* per_shift,
                        void* stream) {
  if (!out) return fail(QMC_EINVAL, "null result pointer");
  cudaStream_t st = (cudaStream_t)stream;
  BatchPlan bp;
  int rc = batch_build(&bp, count, problems, kOneShotWork);
  if (rc == QMC_OK) rc = oneshot_run(&bp, st);
  if (rc == QMC_OK) rc = batch_copy_out(&bp, out, per_shift, st);
  if (bp.ws) {
    cudaFreeAsync(bp.ws, st);
    bp.ws = nullptr;
  }
  cudaError_t e = cudaStreamSynchronize(st);
  if (rc == QMC_OK && e != cudaSuccess) rc = cuda_fail(e, "batch synchronise");
  if (rc == QMC_OK && !is_device_pointer(out))
    for (int i = 0; i < bp.count; ++i)
      if (out[i].status != QMC_OK) return out[i].status;
  return rc;
}

int qmc_integrate_batch_to_tolerance(int32_t count, const qmc_problem* problems, int32_t levels,
                                     const uint64_t* ladder_n, const uint64_t* ladder_g, int32_t ladder_dim,
                                     double rel_tol, int32_t criterion, qmc_result* out, int32_t* level_out,
                                     int32_t* passes_out, void* stream) {
  return batch_walk(count, problems, levels, ladder_n, ladder_g, ladder_dim, rel_tol, criterion, out, level_out,
                    passes_out, (cudaStream_t)stream);
}

int qmc_integrate_batch_extensible(int32_t count, const qmc_problem* problems, int32_t levels, const uint64_t* g,
                                   int32_t g_dim, double rel_tol, int32_t criterion, qmc_result* out,
                                   int32_t* level_out, int32_t* passes_out, void* stream) {
  return batch_extensible(count, problems, levels, g, g_dim, rel_tol, criterion, out, level_out, passes_out,
                          (cudaStream_t)stream);
}

}  // extern "C"

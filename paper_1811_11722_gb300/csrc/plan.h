// Host-side plan of one rule: validated, packed launch descriptors plus the
// device workspace (per-CTA slots, counters, result staging).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "kernel_table.h"
#include "qmc_internal.h"

namespace qmc {

struct SampleIO;

struct Launch {
  const void* func = nullptr;
  void* cufunc = nullptr;  // run-time specialised kernel (CUfunction), if any
  dim3 grid;
  size_t smem = 0;
  std::vector<uint8_t> params;  // kernel parameter struct, passed as args[0]
};

// Launch-shape overrides (autotuner); zero fields mean "library default".
struct TuneChoice {
  int mc = 0;          // shifts per launch chunk (8, 16, 32)
  int L = 0;           // points per thread per tile
  int occupancy = 0;   // cap on CTAs per SM
  bool no_jit = false; // keep the template kernel (no run-time specialisation)
  int max_ctas = 0;    // cap on CTAs of each launch (batched sectors run side by side)
  bool force_general = false;
  int smacc = -1;      // specialised kernel: accumulator pairs in shared memory (1), registers (0),
                       // -1: the QMC_JIT_SMACC default
  int minb = 0;        // specialised kernel: minimum resident CTAs per SM in its launch bounds (0: none)
  int imm = -1;        // specialised kernel: shifts as immediate operands (1), from the launch parameters
                       // (0), -1: the QMC_JIT_IMM default (plans of one launch chunk only)
};

// Deep copy of a problem's host inputs (so a plan can be rebuilt by the tuner).
struct SavedProblem {
  int d = 0;
  uint64_t n = 0;
  int m = 0;
  qmc_transform t{};
  std::vector<uint64_t> g;
  std::vector<double> shifts, cu, cf, c, b;
  std::vector<uint8_t> eu, ef;
  std::vector<int32_t> h;
  qmc_integrand f{};
  qmc_eps eps{};  // orders == 0: no epsilon expansion
  void save(int32_t d_, uint64_t n_, int32_t m_, const uint64_t* g_, const double* shifts_, qmc_transform t_,
            const qmc_integrand* f_);
};

struct Plan {
  int d = 0;
  uint64_t n = 0;
  int m = 0;
  int is_complex = 0;
  int orders = 1;  // result groups: epsilon orders f_0..f_{orders-1}, or integrands + their sum
  bool sum_last = false;  // the last group is the sum of the others (shared-lattice plans)
  int nblk = 0;
  int mc = 0;
  int imm = 0;     // the specialised kernel takes its shifts as immediate operands
  const void* func = nullptr;
  double value_scale = 1.0;
  double final_scale = 1.0;
  double offset[2] = {0.0, 0.0};  // added to Q^(k) per part by the final pass
  std::vector<Launch> launches;
  Workspace ws{};
  void* ws_base = nullptr;
  bool ws_async = false;
  cudaEvent_t ev_before = nullptr;  // optional timing hook
  cudaEvent_t ev_after = nullptr;
  TuneChoice tune{};
  SavedProblem saved;
  // what plan_rebase needs to move the plan to another lattice
  int param_kind = 0;       // launches hold RuleParams<float> (1), RuleParams<double> (2),
                            // GeneralParams<float> (3), GeneralParams<double> (4); 0: fixed lattice
  int grid_occ = 1;         // CTAs per SM the launch shape assumes
  bool grid_capped = true;  // the launch shape honours a cap on CTAs (rule plans; not deformed ones)
};

int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
bool is_device_pointer(const void* p);
bool prime_check(uint64_t n);

int validate_problem(int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts,
                     const qmc_transform& t, const qmc_integrand* f);
int poly_degree(const qmc_poly& p, int d);
bool poly_positive(const qmc_poly& p, int d);
std::vector<double> pack_dense(const qmc_poly& p, int D, int K);
Recip reciprocal(uint64_t n);
void korobov_coefs(int alpha, double* kor);
uint64_t shift_fixed64(double delta);
int choose_grid(const void* func, size_t smem, uint64_t n, int& nblk, int& L, uint64_t& tiles,
                int occupancy_override);
int grid_occupancy(const void* func, size_t smem, int occupancy_override, int& occ);
int grid_shape(int occ, uint64_t n, int max_ctas, int fixed_L, int& nblk, int& L, uint64_t& tiles);
// Move a built plan to the lattice (n, g) of the same dimension: lattice
// fields and launch shape of every launch (max_ctas as TuneChoice::max_ctas);
// kernels, shifts and coefficients are kept.  QMC_EUNSUPPORTED for plans
// whose launches are not rule launches (param_kind 0).
int plan_rebase(Plan* pl, uint64_t n, const uint64_t* g, int max_ctas);
// Give a built plan new shifts [m][d] in [0, 1) (host), encoded as at build
// time; lattice, kernels and coefficients are kept.  QMC_EUNSUPPORTED for
// plans that are not rule plans or have their shifts compiled in.
int plan_reshift(Plan* pl, const double* shifts);

template <typename R>
void fill_common(RuleParams<R>& P, int32_t d, uint64_t n, const uint64_t* g, const qmc_transform& t,
                 const qmc_integrand* f);

int plan_build(Plan* pl, int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts,
               qmc_transform t, const qmc_integrand* f, const TuneChoice& tune, const qmc_eps* eps = nullptr);
int build_deformed_plan(Plan* pl, int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts,
                        const qmc_transform& t, const qmc_integrand* f, const TuneChoice& tune);
int plan_alloc(Plan* pl, cudaStream_t stream, bool async);
void plan_free(Plan* pl, cudaStream_t stream);
int launch_rule(const Plan* pl, const Workspace& ws, cudaStream_t stream, const SampleIO& sio);
int launch_finalize(const Plan* pl, const Workspace& ws, qmc_result* res_dev, double* per_shift_dev,
                    cudaStream_t stream);
int plan_execute(Plan* pl, qmc_result* out, double* per_shift, cudaStream_t stream);

bool jit_enabled();
bool jit_smacc();
bool jit_imm();
int jit_sector_f32(int D, int MC, int TR, int ALPHA, bool check, const std::vector<double>& cu,
                   const std::vector<double>& cf, bool smacc, int minb, void** fn_out, int* occ_out,
                   size_t* smem_out, const uint32_t* imm_shifts = nullptr);
int jit_multi_f32(int D, int MC, int TR, int ALPHA, bool check,
                  const std::vector<std::pair<std::vector<double>, std::vector<double>>>& polys, void** fn_out,
                  int* occ_out);
int jit_eps_f32(int D, int MC, int NE, int TR, int ALPHA, bool log1, bool check, const std::vector<double>& cu,
                const std::vector<double>& cf, void** fn_out, int* occ_out);
// One sector of a run-time specialised persistent batch: its rule as the
// packed FP32 sector path sees it (prescaled dense slots of U and F).
struct PjSector {
  int d = 0, tr = 0;
  bool check = false;
  uint64_t n = 0;
  Recip rc{0, 0};
  uint32_t g[QMC_DMAX] = {0}, gstep[QMC_DMAX] = {0};
  std::vector<double> cu, cf;
  float kor[8] = {0};
};
// One descriptor: a sector and a chunk of shift rows (rows >= m repeat row 0).
struct PjDesc {
  int sector = 0, kbase = 0, m = 0, mc = 0;
  std::vector<uint32_t> shift;  // [mc][d], 32-bit fixed point
};
// Compile (or fetch) the persistent kernel qmc_jit_persist for these
// descriptors (one NVRTC program per group of sectors, compiled on the host
// cores as relocatable code and linked); QMC_OK with the CUfunction and its
// occupancy, else an error code (the caller keeps the generic kernel).
// min_ctas: resident CTAs per SM the kernel is built for (1, or 2 with every
// function held to 128 registers).  runtime_lattice: the kernel (qmc_jit_walk)
// reads each descriptor's lattice and slots from PersistArgs::lats instead of
// compiling the lattice in (the batched ladder walk).
int jit_persist(const std::vector<PjSector>& secs, const std::vector<PjDesc>& descs, int min_ctas, void** fn_out,
                int* occ_out, bool runtime_lattice = false);

int device_sms();
int launch_any(const Launch& ln, dim3 grid, void** args, cudaStream_t stream);
int graph_add_launch(cudaGraph_t graph, const Launch& ln, void** args, cudaGraphNode_t* node,
                     const cudaGraphNode_t* deps = nullptr, size_t ndeps = 0);

}  // namespace qmc

// Run-time specialisation of the FP32 sector kernel for one plan's integrand.
//
// The template kernel reads U and F as dense nested-Horner coefficient
// arrays, so it spends an FMA on every monomial slot whether or not the
// polynomial has that monomial (F with 12 terms in d = 6 still costs 27
// FMAs) plus moves for FMAs whose two constant operands cannot both be
// encoded.  For a given plan the host writes U and F as straight-line code
// that keeps only the nonzero monomials, in the same nesting order, with each
// coefficient an exact hexadecimal float literal, and compiles the kernel
// template around it with NVRTC for sm_103a.  Dropped terms are exact zeros
// (fma(0, z, r) == r), so the specialised kernel returns bit-identical
// results; it only executes fewer instructions.  Both the scalar form (point
// sampling) and the packed two-shift form (the rule) are generated.  Any failure (no NVRTC, an
// architecture it does not know, a compile error) leaves the plan on the
// template kernel.  Compiled modules are cached per process by source text
// and device.
#include <cuda.h>
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <nvrtc.h>

#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "plan.h"

namespace qmc {

namespace {

// Driver API entry points, resolved at run time through the runtime (the
// library does not link libcuda, so it still loads on a machine without a
// GPU driver, where only host-side entry points are usable).
struct DriverApi {
  CUresult (*moduleLoadData)(CUmodule*, const void*) = nullptr;
  CUresult (*moduleUnload)(CUmodule) = nullptr;
  CUresult (*moduleGetFunction)(CUfunction*, CUmodule, const char*) = nullptr;
  CUresult (*launchKernel)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned,
                           CUstream, void**, void**) = nullptr;
  CUresult (*occupancy)(int*, CUfunction, int, size_t) = nullptr;
  CUresult (*graphAddKernelNode)(CUgraphNode*, CUgraph, const CUgraphNode*, size_t,
                                 const CUDA_KERNEL_NODE_PARAMS*) = nullptr;
  CUresult (*getErrorString)(CUresult, const char**) = nullptr;
  CUresult (*funcSetAttribute)(CUfunction, CUfunction_attribute, int) = nullptr;
  // linker of relocatable device code (the specialised persistent batch)
  CUresult (*linkCreate)(unsigned, CUjit_option*, void**, CUlinkState*) = nullptr;
  CUresult (*linkAddData)(CUlinkState, CUjitInputType, void*, size_t, const char*, unsigned, CUjit_option*,
                          void**) = nullptr;
  CUresult (*linkComplete)(CUlinkState, void**, size_t*) = nullptr;
  CUresult (*linkDestroy)(CUlinkState) = nullptr;
  CUresult (*graphAddKernelNodeDeps)(CUgraphNode*, CUgraph, const CUgraphNode*, size_t,
                                     const CUDA_KERNEL_NODE_PARAMS*) = nullptr;
  bool ok = false;
  bool link_ok = false;
};

const DriverApi& driver() {
  static DriverApi api;
  static std::once_flag once;
  std::call_once(once, [] {
    auto get = [](const char* name, void** fn) {
      cudaDriverEntryPointQueryResult q;
      return cudaGetDriverEntryPointByVersion(name, fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
             q == cudaDriverEntryPointSuccess && *fn;
    };
    api.ok = get("cuModuleLoadData", (void**)&api.moduleLoadData) &&
             get("cuModuleUnload", (void**)&api.moduleUnload) &&
             get("cuModuleGetFunction", (void**)&api.moduleGetFunction) &&
             get("cuLaunchKernel", (void**)&api.launchKernel) &&
             get("cuOccupancyMaxActiveBlocksPerMultiprocessor", (void**)&api.occupancy) &&
             get("cuGraphAddKernelNode", (void**)&api.graphAddKernelNode) &&
             get("cuGetErrorString", (void**)&api.getErrorString) &&
             get("cuFuncSetAttribute", (void**)&api.funcSetAttribute);
    api.link_ok = api.ok && get("cuLinkCreate", (void**)&api.linkCreate) &&
                  get("cuLinkAddData", (void**)&api.linkAddData) &&
                  get("cuLinkComplete", (void**)&api.linkComplete) &&
                  get("cuLinkDestroy", (void**)&api.linkDestroy);
    if (!api.ok || !api.link_ok) cudaGetLastError();
  });
  return api;
}

struct JitEntry {
  CUmodule mod = nullptr;
  CUfunction fn = nullptr;
  int occupancy = 0;
};

std::mutex g_jit_mu;
std::map<std::string, JitEntry> g_jit_cache;

std::string lit(double v) {
  char b[64];
  std::snprintf(b, sizeof(b), "%af", (double)(float)v);
  return b;
}

std::string csrc_dir() {
  Dl_info info;
  if (!dladdr((void*)&csrc_dir, &info) || !info.dli_fname) return ".";
  std::string p = info.dli_fname;
  size_t s = p.find_last_of('/');
  return (s == std::string::npos ? std::string(".") : p.substr(0, s)) + "/csrc";
}

// Straight-line U (degree 1) and F (degree 2) from the dense slots, in the
// order poly_dense evaluates them, skipping exact zeros.
std::string poly_code(int D, const std::vector<double>& cu, const std::vector<double>& cf) {
  std::string s;
  s += "    R u = " + lit(cu[0]) + ";\n";
  for (int i = 0; i < D; ++i)
    if ((float)cu[1 + i] != 0.0f) s += "    u = fmaf(" + lit(cu[1 + i]) + ", z[" + std::to_string(i) + "], u);\n";
  s += "    R f = " + lit(cf[0]) + ";\n";
  int off = 1;
  for (int i = 0; i < D; ++i) {
    const double li = cf[off];
    std::string r;
    bool any = (float)li != 0.0f;
    if (any) r = lit(li);
    for (int j = i; j < D; ++j) {
      const double q = cf[off + 1 + (j - i)];
      if ((float)q == 0.0f) continue;
      const std::string zj = "z[" + std::to_string(j) + "]";
      if (!any) {
        r = "(" + lit(q) + " * " + zj + ")";
        any = true;
      } else {
        r = "fmaf(" + lit(q) + ", " + zj + ", " + r + ")";
      }
    }
    if (any) s += "    f = fmaf(z[" + std::to_string(i) + "], " + r + ", f);\n";
    off += 1 + (D - i);
  }
  s += "    U = u;\n    F = f;\n";
  return s;
}

// The packed counterpart (U and -F on coordinate pairs, DensePolys::eval2):
// the same chains over the (c, c) pairs of the kernel parameters, skipping the
// slots whose coefficient is zero.
std::string poly_code2(int D, const std::vector<double>& cu, const std::vector<double>& cf,
                       const std::string& arr = "P.cp", const std::vector<int>* remap = nullptr) {
  auto pc = [&arr, remap](int slot) { return arr + "[" + std::to_string(remap ? (*remap)[slot] : slot) + "]"; };
  const int nu = 1 + D;
  std::string s;
  s += "    float2 u = " + pc(0) + ";\n";
  for (int i = 0; i < D; ++i)
    if ((float)cu[1 + i] != 0.0f) s += "    u = fma2(" + pc(1 + i) + ", z[" + std::to_string(i) + "], u);\n";
  s += "    float2 f = " + pc(nu) + ";\n";
  int off = 1;
  for (int i = 0; i < D; ++i) {
    std::string r;
    bool any = (float)cf[off] != 0.0f;
    if (any) r = pc(nu + off);
    for (int j = i; j < D; ++j) {
      const int slot = off + 1 + (j - i);
      if ((float)cf[slot] == 0.0f) continue;
      const std::string zj = "z[" + std::to_string(j) + "]";
      r = any ? "fma2(" + pc(nu + slot) + ", " + zj + ", " + r + ")" : "mul2(" + pc(nu + slot) + ", " + zj + ")";
      any = true;
    }
    if (any) s += "    f = fma2(z[" + std::to_string(i) + "], " + r + ", f);\n";
    off += 1 + (D - i);
  }
  s += "    U = u;\n    Fn = f;\n";
  return s;
}

}  // namespace

bool jit_enabled() {
  const char* e = std::getenv("QMC_JIT");
  return !(e && e[0] == '0');
}

// Shifts as immediate operands of the specialised kernel (QMC_JIT_IMM=1; launch parameters otherwise).
bool jit_imm() {
  const char* e = std::getenv("QMC_JIT_IMM");
  return e && e[0] == '1';
}

// Accumulator pairs in shared memory for the specialised kernel (QMC_JIT_SMACC=1; registers otherwise).
bool jit_smacc() {
  const char* e = std::getenv("QMC_JIT_SMACC");
  return e && e[0] == '1';
}

// NVRTC-compile `src` for this device (or fetch it from the cache) and
// return kernel `name` with its occupancy at kThreads threads and `smem`
// bytes of dynamic shared memory.  QMC_OK, or an error code (callers fall
// back or report it).
static int jit_compile(const std::string& src, const char* name, size_t smem, void** fn_out, int* occ_out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return QMC_ECUDA;
  }
  const std::string key = std::to_string(dev) + "\n" + src;
  {
    std::lock_guard<std::mutex> lk(g_jit_mu);
    auto it = g_jit_cache.find(key);
    if (it != g_jit_cache.end()) {
      *fn_out = (void*)it->second.fn;
      *occ_out = it->second.occupancy;
      return QMC_OK;
    }
  }
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3) return QMC_EUNSUPPORTED;  // the build targets sm_103a only
  // compile outside the lock (NVRTC programs are independent, so plans can be
  // built on several host threads at once)
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, src.c_str(), "qmc_jit.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
    return QMC_EUNSUPPORTED;
  const std::string inc = "-I" + csrc_dir();
  const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", inc.c_str(), "-lineinfo"};
  nvrtcResult cr = nvrtcCompileProgram(prog, 4, opts);
  if (cr != NVRTC_SUCCESS) {
    size_t ls = 0;
    nvrtcGetProgramLogSize(prog, &ls);
    std::string log(ls, '\0');
    nvrtcGetProgramLog(prog, &log[0]);
    nvrtcDestroyProgram(&prog);
    fail(QMC_EUNSUPPORTED, "run-time specialisation failed to compile: %.400s", log.c_str());
    return QMC_EUNSUPPORTED;
  }
  size_t n = 0;
  nvrtcGetCUBINSize(prog, &n);
  std::vector<char> cubin(n);
  nvrtcGetCUBIN(prog, cubin.data());
  nvrtcDestroyProgram(&prog);
  cudaFree(nullptr);  // make sure the runtime's primary context is current for the driver API
  const DriverApi& drv = driver();
  if (!drv.ok) return QMC_EUNSUPPORTED;
  std::lock_guard<std::mutex> lk(g_jit_mu);
  auto it = g_jit_cache.find(key);  // another thread may have finished the same source
  if (it != g_jit_cache.end()) {
    *fn_out = (void*)it->second.fn;
    *occ_out = it->second.occupancy;
    return QMC_OK;
  }
  JitEntry e;
  if (drv.moduleLoadData(&e.mod, cubin.data()) != CUDA_SUCCESS) return QMC_EUNSUPPORTED;
  if (drv.moduleGetFunction(&e.fn, e.mod, name) != CUDA_SUCCESS) {
    drv.moduleUnload(e.mod);
    return QMC_EUNSUPPORTED;
  }
  if (smem > 48 * 1024 &&
      drv.funcSetAttribute(e.fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, (int)smem) != CUDA_SUCCESS) {
    drv.moduleUnload(e.mod);
    return QMC_EUNSUPPORTED;
  }
  if (drv.occupancy(&e.occupancy, e.fn, kThreads, smem) != CUDA_SUCCESS || e.occupancy < 1) e.occupancy = 1;
  g_jit_cache[key] = e;
  *fn_out = (void*)e.fn;
  *occ_out = e.occupancy;
  return QMC_OK;
}

// The include line and the GenPolys policy (scalar eval for point sampling,
// packed eval2 for the rule, and the packed path's shifts: the launch
// parameters', or, given imm_shifts [MC][D], immediate operands) of one
// integrand.
static std::string gen_polys(int D, const std::vector<double>& cu, const std::vector<double>& cf,
                             const uint32_t* imm_shifts = nullptr, int MC = 0) {
  std::string src;
  src += "#include \"rule_kernels.cuh\"\n";
  src += "namespace qmc {\nstruct GenPolys {\n";
  if (imm_shifts) {
    src += "  __device__ static __forceinline__ uint32_t shift(const RuleParams<float>&, int k, int i) {\n";
    src += "    switch (k * 16 + i) {\n";
    for (int k = 0; k < MC; ++k)
      for (int i = 0; i < D; ++i) {
        char b[80];
        std::snprintf(b, sizeof(b), "      case %d: return 0x%08xu;\n", k * 16 + i, imm_shifts[(size_t)k * D + i]);
        src += b;
      }
    src += "    }\n    return 0u;\n  }\n";
  } else {
    src += "  __device__ static __forceinline__ uint32_t shift(const RuleParams<float>& P, int k, int i) {\n";
    src += "    return P.shiftx[k][i];\n  }\n";
  }
  src += "  template <int D_, int KU, int KF, typename R>\n";
  src += "  __device__ static __forceinline__ void eval(const RuleParams<R>&, const R* z, R& U, R& F) {\n";
  src += poly_code(D, cu, cf);
  src += "  }\n";
  src += "  template <int D_, int KU, int KF>\n";
  src += "  __device__ static __forceinline__ void eval2(const RuleParams<float>& P, const float2* z, float2& U,\n";
  src += "                                               float2& Fn) {\n";
  src += poly_code2(D, cu, cf);
  src += "  }\n};\n}  // namespace qmc\n";
  return src;
}

// Compile (or fetch) the specialised FP32 epsilon-order kernel (eps_body2):
// NE orders, MC shifts per launch, one logarithm per value when log1.
int jit_eps_f32(int D, int MC, int NE, int TR, int ALPHA, bool log1, bool check, const std::vector<double>& cu,
                const std::vector<double>& cf, void** fn_out, int* occ_out) {
  std::string src = gen_polys(D, cu, cf);
  src += "extern \"C\" __global__ void __launch_bounds__(256) qmc_jit_eps(\n";
  src += "    const __grid_constant__ qmc::RuleParams<float> P, double* __restrict__ partial,\n";
  src += "    unsigned long long* __restrict__ counters, const qmc::SampleIO sio) {\n";
  src += "  qmc::eps_body2<" + std::to_string(D) + ", " + std::to_string(MC) + ", " + std::to_string(NE) + ", " +
         std::to_string(TR) + ", " + std::to_string(ALPHA) + ", " + (log1 ? "true" : "false") + ", " +
         (check ? "true" : "false") + ", qmc::GenPolys>(P, partial, counters, sio);\n}\n";
  return jit_compile(src, "qmc_jit_eps", 0, fn_out, occ_out);
}

// Compile (or fetch) the specialised FP32 sector kernel.  Returns QMC_OK and
// the CUfunction / occupancy, or an error code (the caller falls back).
int jit_sector_f32(int D, int MC, int TR, int ALPHA, bool check, const std::vector<double>& cu,
                   const std::vector<double>& cf, bool smacc, int minb, void** fn_out, int* occ_out,
                   size_t* smem_out, const uint32_t* imm_shifts) {
  const size_t smem = smacc ? (size_t)MC * kThreads * 8 : 0;
  *smem_out = smem;
  std::string src = gen_polys(D, cu, cf, imm_shifts, MC);
  src += "extern \"C\" __global__ void __launch_bounds__(256" + (minb > 0 ? ", " + std::to_string(minb) : "") +
         ") qmc_jit_sector(\n";
  src += "    const __grid_constant__ qmc::RuleParams<float> P, double* __restrict__ partial,\n";
  src += "    unsigned long long* __restrict__ counters, const qmc::SampleIO sio) {\n";
  src += "  qmc::sector_body<float, " + std::to_string(D) + ", " + std::to_string(MC) + ", " + std::to_string(TR) +
         ", " + std::to_string(ALPHA) + ", 1, 2, " + (check ? "true" : "false") +
         ", qmc::GenPolys, " + (smacc ? "true" : "false") + ">(P, partial, counters, sio);\n}\n";
  return jit_compile(src, "qmc_jit_sector", smem, fn_out, occ_out);
}

// Compile (or fetch) the shared-lattice kernel for one chunk of integrands:
// polys[s] = (U slots, F slots) of integrand s of the chunk.  Their
// coefficients are read from MultiParams::cps, so chunks whose integrands
// have the same monomials share one compiled kernel.
int jit_multi_f32(int D, int MC, int TR, int ALPHA, bool check,
                  const std::vector<std::pair<std::vector<double>, std::vector<double>>>& polys, void** fn_out,
                  int* occ_out) {
  const int SC = (int)polys.size();
  if (SC < 1 || SC > kMultiChunk) return QMC_EINVAL;
  std::string src;
  src += "#include \"rule_kernels.cuh\"\n";
  src += "namespace qmc {\nstruct GenMulti {\n";
  src += "  __device__ static __forceinline__ void eval2(const MultiParams& M, int s, const float2* z, float2& U,\n";
  src += "                                               float2& Fn) {\n";
  for (int s = 0; s < SC; ++s) {
    src += std::string(s ? "    } else if" : "    if") + " (s == " + std::to_string(s) + ") {\n";
    src += poly_code2(D, polys[s].first, polys[s].second, "M.cps[" + std::to_string(s) + "]");
  }
  src += "    }\n  }\n};\n}  // namespace qmc\n";
  src += "extern \"C\" __global__ void __launch_bounds__(256) qmc_jit_multi(\n";
  src += "    const __grid_constant__ qmc::MultiParams M, double* __restrict__ partial,\n";
  src += "    unsigned long long* __restrict__ counters, const qmc::SampleIO sio) {\n";
  src += "  qmc::multi_body<" + std::to_string(D) + ", " + std::to_string(MC) + ", " + std::to_string(SC) + ", " +
         std::to_string(TR) + ", " + std::to_string(ALPHA) + ", " + (check ? "true" : "false") +
         ", qmc::GenMulti>(M, partial, counters);\n}\n";
  return jit_compile(src, "qmc_jit_multi", 0, fn_out, occ_out);
}

// ---------------------------------------------- specialised persistent batch --

namespace {

std::string hex32(uint32_t v) {
  char b[24];
  std::snprintf(b, sizeof(b), "0x%08xu", v);
  return b;
}
std::string hex64(uint64_t v) {
  char b[32];
  std::snprintf(b, sizeof(b), "0x%016llxull", (unsigned long long)v);
  return b;
}

// Pair slots (U's then -F's, the order of fill_pairs) that poly_code2 reads:
// the constant terms and every slot with a nonzero coefficient.  remap[slot]
// is the slot's index in the compact array, -1 if unused.
std::vector<int> used_pairs(const PjSector& S, std::vector<float>* vals) {
  const int nu = 1 + S.d;
  const int nf = (int)S.cf.size();
  std::vector<int> remap(nu + nf, -1);
  int c = 0;
  auto take = [&](int slot, float v) {
    remap[slot] = c++;
    vals->push_back(v);
  };
  take(0, (float)S.cu[0]);
  for (int i = 0; i < S.d; ++i)
    if ((float)S.cu[1 + i] != 0.0f) take(1 + i, (float)S.cu[1 + i]);
  take(nu, -(float)S.cf[0]);
  for (int t = 1; t < nf; ++t)
    if ((float)S.cf[t] != 0.0f) take(nu + t, -(float)S.cf[t]);
  return remap;
}

// One NVRTC program compiled as relocatable device code (every function held
// to max_regs registers); its CUBIN in *out.
int nvrtc_rdc(const std::string& src, const std::string& name, int max_regs, std::vector<char>* out,
              std::string* log) {
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, src.c_str(), name.c_str(), 0, nullptr, nullptr) != NVRTC_SUCCESS)
    return QMC_EUNSUPPORTED;
  const std::string inc = "-I" + csrc_dir();
  const std::string regs = "--maxrregcount=" + std::to_string(max_regs);
  const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", inc.c_str(), "-lineinfo",
                        "--relocatable-device-code=true", regs.c_str()};
  nvrtcResult cr = nvrtcCompileProgram(prog, 6, opts);
  if (cr != NVRTC_SUCCESS) {
    size_t ls = 0;
    nvrtcGetProgramLogSize(prog, &ls);
    log->assign(ls, '\0');
    nvrtcGetProgramLog(prog, &(*log)[0]);
    nvrtcDestroyProgram(&prog);
    return QMC_EUNSUPPORTED;
  }
  size_t n = 0;
  nvrtcGetCUBINSize(prog, &n);
  out->resize(n);
  nvrtcGetCUBIN(prog, out->data());
  nvrtcDestroyProgram(&prog);
  return QMC_OK;
}

}  // namespace

// The sources of the specialised persistent module: one program per group of
// sectors (their coefficient pairs, one struct and one device function per
// descriptor) and the dispatching kernel.  QMC_EUNSUPPORTED when the nonzero
// coefficient pairs exceed what the module's constant bank holds.
int persist_sources(const std::vector<PjSector>& secs, const std::vector<PjDesc>& descs, int ngroups, int min_ctas,
                    bool rt, std::vector<std::string>* gsrc_out, std::string* msrc_out) {
  const int nsec = (int)secs.size();
  std::vector<std::string>& gsrc = *gsrc_out;
  gsrc.assign(ngroups, std::string());
  std::vector<std::vector<int>> remaps(nsec);
  size_t const_bytes = 0;
  for (int g = 0; g < ngroups; ++g) {
    std::string& src = gsrc[g];
    src += "#include \"persist_jit.cuh\"\n";
    src += "__constant__ float qmc_kor_g" + std::to_string(g) + "[8] = {";
    for (int k = 0; k < 8; ++k) src += (k ? ", " : "") + lit(secs[0].kor[k]);
    src += "};\n";
  }
  for (int s = 0; s < nsec; ++s) {
    const PjSector& S = secs[s];
    std::vector<float> vals;
    remaps[s] = used_pairs(S, &vals);
    const_bytes += vals.size() * 8;
    std::string& src = gsrc[s % ngroups];
    src += "__constant__ float2 qmc_cp_s" + std::to_string(s) + "[" + std::to_string(vals.size()) + "] = {";
    for (size_t q = 0; q < vals.size(); ++q) src += (q ? ", {" : "{") + lit(vals[q]) + ", " + lit(vals[q]) + "}";
    src += "};\n";
  }
  if (const_bytes > 60 * 1024) return QMC_EUNSUPPORTED;  // the constant bank of one module holds 64 KB
  for (size_t q = 0; q < descs.size(); ++q) {
    const PjDesc& Dq = descs[q];
    const PjSector& S = secs[Dq.sector];
    const int g = Dq.sector % ngroups;
    std::string& src = gsrc[g];
    const std::string nm = "qmc_sp_" + std::to_string(q);
    src += "struct " + nm + " {\n";
    src += "  static constexpr int D = " + std::to_string(S.d) + ", TR = " + std::to_string(S.tr) +
           ", ALPHA = " + std::to_string(S.tr == TR_KOROBOV ? 3 : 0) + ", MC = " + std::to_string(Dq.mc) +
           ", M = " + std::to_string(Dq.m) + ", KBASE = " + std::to_string(Dq.kbase) + ";\n";
    src += std::string("  static constexpr bool CHECK = ") + (S.check ? "true" : "false") + ";\n";
    if (!rt) {  // the lattice as constants (with run-time lattices it comes from the launch)
      src += "  static constexpr unsigned long long N = " + hex64(S.n) + ", RHI = " + hex64(S.rc.rhi) +
             ", RLO = " + hex64(S.rc.rlo) + ";\n";
      auto table = [&](const char* fname, int count, auto value) {
        src += std::string("  __device__ static __forceinline__ unsigned ") + fname + "(int i) {\n    switch (i) {\n";
        for (int c = 0; c < count; ++c) src += "      case " + std::to_string(c) + ": return " + value(c) + ";\n";
        src += "    }\n    return 0u;\n  }\n";
      };
      table("g", S.d, [&](int i) { return hex32(S.g[i]); });
      table("gstep", S.d, [&](int i) { return hex32(S.gstep[i]); });
    }
    {
      src += "  __device__ static __forceinline__ unsigned shift(int k, int i) {\n    switch (k * 16 + i) {\n";
      for (int k = 0; k < Dq.mc; ++k)
        for (int i = 0; i < S.d; ++i)
          src += "      case " + std::to_string(k * 16 + i) + ": return " + hex32(Dq.shift[(size_t)k * S.d + i]) + ";\n";
      src += "    }\n    return 0u;\n  }\n";
    }
    src += "  __device__ static __forceinline__ const float* kor() { return qmc_kor_g" + std::to_string(g) + "; }\n";
    src += "  __device__ static __forceinline__ void eval2(const float2* z, float2& U, float2& Fn) {\n";
    src += "    using namespace qmc;\n";
    src += poly_code2(S.d, S.cu, S.cf, "qmc_cp_s" + std::to_string(Dq.sector), &remaps[Dq.sector]);
    src += "  }\n};\n";
    src += "extern \"C\" __device__ void qmc_pd_" + std::to_string(q) +
           "(unsigned long long j0, unsigned long long chunk, unsigned item, int nitems, double* partial, "
           "unsigned long long* counters, double (*red)[qmc::kPjMc], const qmc::PjLattice* lat) {\n";
    src += "  qmc::pj_sweep<" + nm + (rt ? ", true" : ", false") +
           ">(j0, chunk, item, nitems, partial, counters, red, lat);\n}\n";
  }
  std::string& msrc = *msrc_out;
  msrc = "#include \"persist_jit.cuh\"\n";
  for (size_t q = 0; q < descs.size(); ++q)
    msrc += "extern \"C\" __device__ void qmc_pd_" + std::to_string(q) +
            "(unsigned long long, unsigned long long, unsigned, int, double*, unsigned long long*, "
            "double (*)[qmc::kPjMc], const qmc::PjLattice*);\n";
  msrc +=
      "extern \"C\" __global__ void __launch_bounds__(256, " + std::to_string(min_ctas) + ") " +
      std::string(rt ? "qmc_jit_walk" : "qmc_jit_persist") +
      "(const __grid_constant__ qmc::PersistArgs A) {\n"
      "  __shared__ double red[qmc::kThreads / 32][qmc::kPjMc];\n"
      "  __shared__ unsigned cur;\n"
      "  for (;;) {\n"
      "    if (threadIdx.x == 0) cur = atomicAdd(A.next, 1u);\n"
      "    __syncthreads();\n"
      "    const unsigned it = cur;\n"
      "    if (it >= A.nitems) break;  // the same for every thread of the CTA\n"
      "    const qmc::PersistItem wi = A.items[it];\n"
      "    const unsigned long long j0 = (unsigned long long)wi.item * A.chunk;\n";
  if (rt)
    msrc +=
        "    const qmc::PjLattice* lat = A.lats + wi.desc;\n"
        "    double* partial = lat->partial;\n"
        "    unsigned long long* counters = lat->counters;\n"
        "    const int nitems = lat->nitems;\n";
  else
    msrc +=
        "    const qmc::PersistDesc* ds = A.descs + wi.desc;\n"
        "    const qmc::PjLattice* lat = nullptr;\n"
        "    double* partial = ds->partial;\n"
        "    unsigned long long* counters = ds->counters;\n"
        "    const int nitems = ds->nitems;\n";
  msrc += "    switch (wi.desc) {\n";
  for (size_t q = 0; q < descs.size(); ++q)
    msrc += "      case " + std::to_string(q) + ": qmc_pd_" + std::to_string(q) +
            "(j0, A.chunk, wi.item, nitems, partial, counters, red, lat); break;\n";
  msrc +=
      "    }\n"
      "    __syncthreads();  // red and cur are rewritten for the next item\n"
      "  }\n}\n";
  return QMC_OK;
}

int jit_persist(const std::vector<PjSector>& secs, const std::vector<PjDesc>& descs, int min_ctas, void** fn_out,
                int* occ_out, bool runtime_lattice) {
  if (secs.empty() || descs.empty() || min_ctas < 1 || min_ctas > 2) return QMC_EINVAL;
  const int max_regs = min_ctas == 2 ? 128 : 255;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return QMC_ECUDA;
  }
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3) return QMC_EUNSUPPORTED;
  // group the sectors (with all of their descriptors) for compilation on the host cores
  const int ngroups = std::max(1, std::min<int>((int)secs.size(),
                                                std::min(32u, std::max(1u, std::thread::hardware_concurrency()))));
  std::vector<std::string> gsrc;
  std::string msrc;
  int rc = persist_sources(secs, descs, ngroups, min_ctas, runtime_lattice, &gsrc, &msrc);
  if (rc) return rc;
  std::string key = std::to_string(dev) + "\npersist " + std::to_string(max_regs) + "\n" + msrc;
  for (const std::string& g : gsrc) key += g;
  {
    std::lock_guard<std::mutex> lk(g_jit_mu);
    auto it = g_jit_cache.find(key);
    if (it != g_jit_cache.end()) {
      *fn_out = (void*)it->second.fn;
      *occ_out = it->second.occupancy;
      return QMC_OK;
    }
  }
  const DriverApi& drv = driver();
  if (!drv.ok || !drv.link_ok) return QMC_EUNSUPPORTED;
  // compile the groups and the dispatching kernel on the host cores
  std::vector<std::vector<char>> cubins(ngroups + 1);
  std::vector<int> rcs(ngroups + 1, QMC_OK);
  std::vector<std::string> logs(ngroups + 1);
  {
    std::vector<std::thread> th;
    for (int g = 0; g <= ngroups; ++g)
      th.emplace_back([&, g]() {
        rcs[g] = g < ngroups ? nvrtc_rdc(gsrc[g], "qmc_persist_g" + std::to_string(g) + ".cu", max_regs, &cubins[g],
                                         &logs[g])
                             : nvrtc_rdc(msrc, "qmc_persist_main.cu", max_regs, &cubins[g], &logs[g]);
      });
    for (auto& t : th) t.join();
  }
  for (int g = 0; g <= ngroups; ++g)
    if (rcs[g] != QMC_OK) {
      fail(QMC_EUNSUPPORTED, "persistent batch specialisation failed to compile: %.400s", logs[g].c_str());
      return QMC_EUNSUPPORTED;
    }
  cudaFree(nullptr);  // the runtime's primary context is current for the driver API
  CUlinkState ls;
  if (drv.linkCreate(0, nullptr, nullptr, &ls) != CUDA_SUCCESS) return QMC_EUNSUPPORTED;
  for (int g = 0; g <= ngroups; ++g) {
    const std::string nm = "qmc_persist_" + std::to_string(g) + ".cubin";
    if (drv.linkAddData(ls, CU_JIT_INPUT_CUBIN, cubins[g].data(), cubins[g].size(), nm.c_str(), 0, nullptr,
                        nullptr) != CUDA_SUCCESS) {
      drv.linkDestroy(ls);
      return QMC_EUNSUPPORTED;
    }
  }
  void* image = nullptr;
  size_t image_size = 0;
  if (drv.linkComplete(ls, &image, &image_size) != CUDA_SUCCESS) {
    drv.linkDestroy(ls);
    return QMC_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_jit_mu);
  JitEntry e;
  const bool loaded = drv.moduleLoadData(&e.mod, image) == CUDA_SUCCESS;
  drv.linkDestroy(ls);  // owns the linked image; the module keeps its own copy
  if (!loaded) return QMC_EUNSUPPORTED;
  if (drv.moduleGetFunction(&e.fn, e.mod, runtime_lattice ? "qmc_jit_walk" : "qmc_jit_persist") != CUDA_SUCCESS) {
    drv.moduleUnload(e.mod);
    return QMC_EUNSUPPORTED;
  }
  if (drv.occupancy(&e.occupancy, e.fn, kThreads, 0) != CUDA_SUCCESS || e.occupancy < 1) e.occupancy = 1;
  g_jit_cache[key] = e;
  *fn_out = (void*)e.fn;
  *occ_out = e.occupancy;
  return QMC_OK;
}

// Launch either a runtime kernel (ln.func) or a specialised one (ln.cufunc).
int launch_any(const Launch& ln, dim3 grid, void** args, cudaStream_t stream) {
  if (ln.cufunc) {
    const DriverApi& drv = driver();
    CUresult r = drv.launchKernel((CUfunction)ln.cufunc, grid.x, grid.y, grid.z, kThreads, 1, 1, (unsigned)ln.smem,
                                  (CUstream)stream, args, nullptr);
    if (r != CUDA_SUCCESS) {
      const char* msg = nullptr;
      drv.getErrorString(r, &msg);
      return fail(QMC_ECUDA, "cuLaunchKernel: %s", msg ? msg : "?");
    }
    return QMC_OK;
  }
  cudaError_t e = cudaLaunchKernel(ln.func, grid, dim3(kThreads), args, 0, stream);
  if (e != cudaSuccess) return cuda_fail(e, "cudaLaunchKernel");
  return QMC_OK;
}

// Kernel node for either kind of launch.
int graph_add_launch(cudaGraph_t graph, const Launch& ln, void** args, cudaGraphNode_t* node,
                     const cudaGraphNode_t* deps, size_t ndeps) {
  if (ln.cufunc) {
    CUDA_KERNEL_NODE_PARAMS kp;
    std::memset(&kp, 0, sizeof(kp));
    kp.func = (CUfunction)ln.cufunc;
    kp.gridDimX = ln.grid.x;
    kp.gridDimY = ln.grid.y;
    kp.gridDimZ = ln.grid.z;
    kp.blockDimX = kThreads;
    kp.blockDimY = 1;
    kp.blockDimZ = 1;
    kp.sharedMemBytes = (unsigned)ln.smem;
    kp.kernelParams = args;
    CUgraphNode n;
    if (driver().graphAddKernelNode(&n, (CUgraph)graph, (const CUgraphNode*)deps, ndeps, &kp) != CUDA_SUCCESS)
      return fail(QMC_ECUDA, "cuGraphAddKernelNode");
    *node = (cudaGraphNode_t)n;
    return QMC_OK;
  }
  cudaKernelNodeParams kp;
  std::memset(&kp, 0, sizeof(kp));
  kp.func = (void*)ln.func;
  kp.gridDim = ln.grid;
  kp.blockDim = dim3(kThreads);
  kp.kernelParams = args;
  cudaError_t e = cudaGraphAddKernelNode(node, graph, deps, ndeps, &kp);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphAddKernelNode");
  return QMC_OK;
}

}  // namespace qmc

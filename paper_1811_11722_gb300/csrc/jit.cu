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
#include <map>
#include <mutex>
#include <string>
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
  bool ok = false;
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
    if (!api.ok) cudaGetLastError();
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
                       const std::string& arr = "P.cp") {
  auto pc = [&arr](int slot) { return arr + "[" + std::to_string(slot) + "]"; };
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
// packed eval2 for the rule) of one integrand.
static std::string gen_polys(int D, const std::vector<double>& cu, const std::vector<double>& cf) {
  std::string src;
  src += "#include \"rule_kernels.cuh\"\n";
  src += "namespace qmc {\nstruct GenPolys {\n";
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
                   size_t* smem_out) {
  const size_t smem = smacc ? (size_t)MC * kThreads * 8 : 0;
  *smem_out = smem;
  std::string src = gen_polys(D, cu, cf);
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
int graph_add_launch(cudaGraph_t graph, const Launch& ln, void** args, cudaGraphNode_t* node) {
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
    if (driver().graphAddKernelNode(&n, (CUgraph)graph, nullptr, 0, &kp) != CUDA_SUCCESS)
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
  cudaError_t e = cudaGraphAddKernelNode(node, graph, nullptr, 0, &kp);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphAddKernelNode");
  return QMC_OK;
}

}  // namespace qmc

// Several integrands on one lattice: one sweep over (point, shift) for all
// sectors of one dimension that share (n, g, shifts, transform), Eq. (2) for
// each and for their sum, Eq. (3) per result.
//
// The fused kernel (multi_body) is specialised at run time for each chunk of
// up to kMultiChunk integrands: their U and -F are straight-line packed
// chains over the nonzero monomials, the coefficients read as (c, c) pairs
// from the launch parameters.  Launches: one per (shift chunk, integrand
// chunk); all use the same grid, so the final pass sees one slot layout
// [integrand][shift][CTA] and forms the sum group from it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <thread>
#include <vector>

#include "plan.h"

namespace qmc {

namespace {

constexpr int kMultiMc = 2;  // shifts per launch: SC x MC run sums stay in registers

int build_multi_plan(Plan* pl, int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts,
                     const qmc_transform& t, int32_t count, const qmc_integrand* fs) {
  if (count < 1 || count > QMC_MULTI_MAX || !fs)
    return fail(QMC_EINVAL, "integrand count %d outside [1, %d]", count, QMC_MULTI_MAX);
  bool check = false;
  for (int s = 0; s < count; ++s) {
    const qmc_integrand& f = fs[s];
    int rc = validate_problem(d, n, m, g, shifts, t, &f);
    if (rc) return rc;
    if (f.kind != QMC_F_SECTOR) return fail(QMC_EINVAL, "integrand %d: shared-lattice sweeps take SECTOR integrands", s);
    if (f.precision != QMC_FP32EVAL || d > kDFast || f.aU != -2 || f.aF != -1 || poly_degree(f.U, d) > 1 ||
        poly_degree(f.F, d) > 2)
      return fail(QMC_EUNSUPPORTED,
                  "integrand %d: the shared-lattice kernel takes FP32EVAL U^-2 F^-1, deg U <= 1, deg F <= 2, d <= %d", s,
                  kDFast);
    if (!poly_positive(f.U, d) || !poly_positive(f.F, d)) check = true;
  }
  const bool kor3 = t.kind == QMC_TRANSFORM_KOROBOV && t.alpha == 3;
  if (t.kind == QMC_TRANSFORM_KOROBOV && !kor3)
    return fail(QMC_EUNSUPPORTED, "shared-lattice kernel: Korobov weight 3 only");
  if (!jit_enabled()) return fail(QMC_EUNSUPPORTED, "shared-lattice kernel needs run-time specialisation (QMC_JIT=0)");

  RuleParams<float> base;
  fill_common(base, d, n, g, t, &fs[0]);
  base.m_total = m;
  const int TR = base.tr, ALPHA = kor3 ? 3 : 0;
  // dense slots of every integrand
  std::vector<std::pair<std::vector<double>, std::vector<double>>> polys(count);
  for (int s = 0; s < count; ++s) {
    polys[s] = {pack_dense(fs[s].U, d, 1), pack_dense(fs[s].F, d, 2)};
    prescale_slots(polys[s].first.data(), d, 1, fx_sigma(TR));  // coordinates arrive divided by fx_sigma
    prescale_slots(polys[s].second.data(), d, 2, fx_sigma(TR));
  }
  // one specialised kernel per integrand chunk, compiled on all host cores
  const int chunks = (count + kMultiChunk - 1) / kMultiChunk;
  std::vector<void*> fn(chunks, nullptr);
  std::vector<int> occ(chunks, 0), rcs(chunks, QMC_OK);
  auto compile = [&](int c) {
    const int s0 = c * kMultiChunk, s1 = std::min(count, s0 + kMultiChunk);
    std::vector<std::pair<std::vector<double>, std::vector<double>>> part(polys.begin() + s0, polys.begin() + s1);
    rcs[c] = jit_multi_f32(d, kMultiMc, TR, ALPHA, check, part, &fn[c], &occ[c]);
  };
  {
    const int hw = std::max(1u, std::thread::hardware_concurrency());
    std::vector<std::thread> pool;
    for (int w = 0; w < std::min(hw, chunks); ++w)
      pool.emplace_back([&, w] {
        for (int c = w; c < chunks; c += std::min(hw, chunks)) compile(c);
      });
    for (auto& th : pool) th.join();
  }
  int min_occ = 1 << 30;
  for (int c = 0; c < chunks; ++c) {
    if (rcs[c])
      return fail(rcs[c], "shared-lattice kernel: run-time specialisation of integrands %d.. failed",
                  c * kMultiChunk);
    min_occ = std::min(min_occ, occ[c]);
  }
  // one resident wave of the least occupied chunk kernel, the same for all launches
  const int sms = device_sms();
  if (sms <= 0) return fail(QMC_ECUDA, "no CUDA device");
  const uint64_t want = (uint64_t)sms * (uint64_t)std::max(1, min_occ);
  const uint64_t per = (n + want * kThreads - 1) / (want * kThreads);
  const int L = (int)std::max<uint64_t>(1, std::min<uint64_t>(per, 512));
  const uint64_t tiles = (n + (uint64_t)kThreads * L - 1) / ((uint64_t)kThreads * L);
  const int nblk = (int)std::min<uint64_t>(want, tiles);
  base.L = L;
  base.tiles = tiles;
  base.nblk = nblk;
  pl->d = d;
  pl->n = n;
  pl->m = m;
  pl->is_complex = 0;
  pl->orders = count + 1;
  pl->sum_last = true;
  pl->nblk = nblk;
  pl->mc = kMultiMc;
  pl->func = nullptr;
  pl->value_scale = 1.0;
  pl->final_scale = base.tr == TR_KOROBOV ? std::pow((double)base.kor[7], (double)d) : 1.0;
  for (int k0 = 0; k0 < m; k0 += kMultiMc) {
    const int mk = std::min(kMultiMc, m - k0);
    for (int c = 0; c < chunks; ++c) {
      std::unique_ptr<MultiParams> M(new MultiParams());
      std::memset(M.get(), 0, sizeof(MultiParams));
      M->base = base;
      M->base.m_launch = mk;
      M->base.k_base = k0;
      for (int kk = 0; kk < kMultiMc; ++kk)  // rows mk.. repeat row k0 (evaluated, never written back)
        for (int i = 0; i < d; ++i) {
          const int src = kk < mk ? k0 + kk : k0;
          set_shift(M->base, kk, i, shift_fixed64(shifts[(size_t)src * d + i]));
        }
      M->s_base = c * kMultiChunk;
      M->count = count;
      const int s1 = std::min(count, M->s_base + kMultiChunk);
      for (int s = M->s_base; s < s1; ++s) {
        const std::vector<double>& cu = polys[s].first;
        const std::vector<double>& cf = polys[s].second;
        const int nu = (int)cu.size();
        for (int q = 0; q < nu; ++q) M->cps[s - M->s_base][q] = make_float2((float)cu[q], (float)cu[q]);
        for (size_t q = 0; q < cf.size(); ++q)
          M->cps[s - M->s_base][nu + q] = make_float2(-(float)cf[q], -(float)cf[q]);
      }
      Launch ln;
      ln.func = nullptr;
      ln.cufunc = fn[c];
      ln.smem = 0;
      ln.grid = dim3(nblk);
      ln.params.resize(sizeof(MultiParams));
      std::memcpy(ln.params.data(), M.get(), sizeof(MultiParams));
      pl->launches.push_back(std::move(ln));
    }
  }
  return QMC_OK;
}

}  // namespace

}  // namespace qmc

using namespace qmc;

extern "C" {

int qmc_multi_plan_create(int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts, qmc_transform t,
                          int32_t count, const qmc_integrand* fs, qmc_plan* plan_out) {
  if (!plan_out) return fail(QMC_EINVAL, "null plan_out");
  *plan_out = nullptr;
  std::unique_ptr<Plan> pl(new Plan());
  int rc = build_multi_plan(pl.get(), d, n, m, g, shifts, t, count, fs);
  if (rc) return rc;
  rc = plan_alloc(pl.get(), nullptr, false);
  if (rc) return rc;
  *plan_out = reinterpret_cast<qmc_plan>(pl.release());
  return QMC_OK;
}

int qmc_integrate_multi(int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts, qmc_transform t,
                        int32_t count, const qmc_integrand* fs, qmc_result* out, double* per_shift, void* stream) {
  Plan pl;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = build_multi_plan(&pl, d, n, m, g, shifts, t, count, fs);
  if (rc) return rc;
  rc = plan_alloc(&pl, s, true);
  if (rc) return rc;
  rc = plan_execute(&pl, out, per_shift, s);
  plan_free(&pl, s);
  return rc;
}

}  // extern "C"

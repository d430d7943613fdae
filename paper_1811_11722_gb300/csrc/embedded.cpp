// Embedded (extensible) rank-1 lattices in base 2, for growing n without
// discarding earlier work.
//
// With N = 2^K and one generating vector g, the lattice of size 2^k uses the
// points J = j 2^(K-k) of the size-N lattice: {j g / 2^k} = {J g / N}.  The
// point sets are nested, and the points of size 2n that are not in size n
// form the size-n lattice shifted by g / (2n).  A rule can therefore double n
// by evaluating one more size-n rule and averaging it, shift by shift, with
// the previous level (qmc_integrate_extensible).
//
// The vector is built component by component as in the CBC search for one n
// (same space and weights, e^2_k = -1 + 2^-k sum_{J : 2^(K-k) | J} prod_i
// (1 + gamma_i B2({J g_i / N}))), choosing each component to minimise the
// worst scaled error over the embedded sizes, max_k 4^k e^2_k.  The e^2 of a
// good lattice decays roughly like n^-2, so the scaling keeps every size in
// play.  The candidates for a component are the odd z in [1, N/2) (z and
// N - z give the same errors; even z would not be units mod 2^k), all of them
// or a SplitMix64-drawn subset.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <thread>
#include <vector>

#include "plan.h"

namespace qmc {

namespace {

inline double bern2(double t) { return t * t - t + 1.0 / 6.0; }

uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// max_k 4^k e^2_k for the vector so far (products p over the N points)
// extended by component z with weight gamma.
double embedded_criterion(const std::vector<double>& p, int K, int kmin, uint64_t z, double gamma) {
  const uint64_t N = 1ull << K;
  // sums of the terms by the number of trailing zero bits of J (J = 0 in every level)
  std::vector<double> bucket(K + 1, 0.0);
  for (uint64_t J = 0; J < N; ++J) {
    const uint64_t r = (J * z) & (N - 1);
    const double term = p[J] * (1.0 + gamma * bern2((double)r / (double)N));
    const int v = J == 0 ? K : std::min(K, __builtin_ctzll(J));
    bucket[v] += term;
  }
  double worst = -1e300, level_sum = 0.0;
  for (int k = 0; k <= K; ++k) {  // level k holds the J with at least K - k trailing zeros
    level_sum += bucket[K - k];
    if (k < kmin) continue;
    const double e2 = level_sum / (double)(1ull << k) - 1.0;
    worst = std::max(worst, std::ldexp(e2, 2 * k));
  }
  return worst;
}

}  // namespace

}  // namespace qmc

using namespace qmc;

extern "C" int qmc_make_lattice_embedded(int32_t d, int32_t log2_nmin, int32_t log2_nmax, const double* gamma,
                                         int32_t candidates, uint64_t seed, uint64_t* g_out) {
  if (d < 1 || d > QMC_DMAX) return fail(QMC_EINVAL, "d=%d outside [1, %d]", d, QMC_DMAX);
  if (log2_nmin < 1 || log2_nmax < log2_nmin || log2_nmax > 30)
    return fail(QMC_EINVAL, "embedded sizes 2^%d..2^%d: need 1 <= min <= max <= 30", log2_nmin, log2_nmax);
  if (!gamma || !g_out || candidates < 1) return fail(QMC_EINVAL, "null weights/output or no candidates");
  for (int i = 0; i < d; ++i)
    if (!(gamma[i] > 0.0) || !std::isfinite(gamma[i])) return fail(QMC_EINVAL, "gamma[%d] must be positive", i);
  const int K = log2_nmax;
  const uint64_t N = 1ull << K;
  std::vector<double> p(N, 1.0);
  auto extend = [&](uint64_t z, double gam) {
    for (uint64_t J = 0; J < N; ++J) p[J] *= 1.0 + gam * bern2((double)((J * z) & (N - 1)) / (double)N);
  };
  g_out[0] = 1;
  extend(1, gamma[0]);
  const uint64_t odd_count = N / 4 > 0 ? N / 4 : 1;  // odd z in [1, N/2)
  for (int s = 1; s < d; ++s) {
    std::vector<uint64_t> cand;
    if ((uint64_t)candidates >= odd_count) {
      for (uint64_t z = 1; z < std::max<uint64_t>(N / 2, 2); z += 2) cand.push_back(z);
    } else {
      uint64_t st = seed ^ (0xD1B54A32D192ED03ull * (uint64_t)(s + 1));
      while ((int)cand.size() < candidates) {
        const uint64_t z = 2 * (splitmix64(st) % odd_count) + 1;
        if (std::find(cand.begin(), cand.end(), z) == cand.end()) cand.push_back(z);
      }
      std::sort(cand.begin(), cand.end());
    }
    std::vector<double> crit(cand.size());
    const unsigned nt = std::max(1u, std::min<unsigned>(64u, std::thread::hardware_concurrency()));
    std::vector<std::thread> th;
    for (unsigned w = 0; w < nt; ++w)
      th.emplace_back([&, w] {
        for (size_t c = w; c < cand.size(); c += nt) crit[c] = embedded_criterion(p, K, log2_nmin, cand[c], gamma[s]);
      });
    for (auto& x : th) x.join();
    size_t best = 0;
    for (size_t c = 1; c < cand.size(); ++c)
      if (crit[c] < crit[best]) best = c;  // strict: ties go to the smaller z
    g_out[s] = cand[best];
    extend(cand[best], gamma[s]);
  }
  return QMC_OK;
}

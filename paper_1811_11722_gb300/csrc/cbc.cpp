// Generating-vector construction for the rank-1 lattice of Eq. (2).
//
// The paper takes g as an input; this is the standard component-by-component
// (CBC) search of the QMC review it cites: with g_1 = 1, component s is the
// candidate z in [1, (n-1)/2] minimising the shift-averaged worst-case error
// in the unanchored weighted Sobolev space with product weights,
//   e^2 = -1 + (1/n) sum_{k=0}^{n-1} prod_{i<=s} (1 + gamma_i B2({k g_i / n})),
//   B2(t) = t^2 - t + 1/6.
// For prime n, ordering both k and z by powers of a primitive root w turns the
// candidate-by-point matrix B2({k z / n}) into a circulant of length n - 1
// (Nuyens and Cools, Math. Comp. 75, 2006); since B2 is symmetric about 1/2
// and w^((n-1)/2) = -1 it even has period h = (n-1)/2.  All candidates of one
// component then come from one cyclic convolution of length h, done here as a
// zero-padded power-of-two complex FFT on the host cores (O(n log n) per
// component instead of O(n^2)).  The FFT's rounding noise (~1e-16 n) can
// exceed the gaps between the best candidates at large n, so the kRerank
// candidates with the smallest convolution values are re-evaluated exactly,
//   T(z) = sum_{k=0}^{n-1} p[k] B2({k z / n})   (Neumaier, k ascending),
// and the smallest T wins (ties to the smallest z).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <functional>
#include <thread>
#include <vector>

#include "plan.h"

namespace qmc {

using cd = std::complex<double>;

static void parallel_for(size_t n, const std::function<void(size_t, size_t)>& body) {
  unsigned nt = std::max(1u, std::min(64u, std::thread::hardware_concurrency()));
  if (n < (1u << 16) || nt == 1) {
    body(0, n);
    return;
  }
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nt; ++t) {
    size_t a = n * t / nt, b = n * (t + 1) / nt;
    th.emplace_back([=, &body] { body(a, b); });
  }
  for (auto& x : th) x.join();
}

// In-place iterative radix-2 FFT, sign -1 forward, +1 inverse (unscaled).
// tw[k] = exp(-2 pi i k / M) for k < M/2.
static void fft(std::vector<cd>& a, const std::vector<cd>& tw, int logM, bool inverse) {
  const size_t M = (size_t)1 << logM;
  parallel_for(M, [&](size_t lo, size_t hi) {
    for (size_t i = lo; i < hi; ++i) {
      size_t r = 0, x = i;
      for (int b = 0; b < logM; ++b) {
        r = (r << 1) | (x & 1);
        x >>= 1;
      }
      if (i < r) std::swap(a[i], a[r]);
    }
  });
  for (int s = 1; s <= logM; ++s) {
    const size_t half = (size_t)1 << (s - 1), len = half << 1, stride = M / len;
    parallel_for(M / 2, [&](size_t lo, size_t hi) {
      for (size_t b = lo; b < hi; ++b) {
        size_t blk = b / half, k = b % half;
        size_t i = blk * len + k, j = i + half;
        cd w = tw[k * stride];
        if (inverse) w = std::conj(w);
        cd t = a[j] * w;
        a[j] = a[i] - t;
        a[i] += t;
      }
    });
  }
}

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t n) { return (uint64_t)((unsigned __int128)a * b % n); }

static uint64_t powmod(uint64_t a, uint64_t e, uint64_t n) {
  uint64_t r = 1;
  while (e) {
    if (e & 1) r = mulmod(r, a, n);
    a = mulmod(a, a, n);
    e >>= 1;
  }
  return r;
}

static uint64_t primitive_root(uint64_t n) {
  std::vector<uint64_t> fac;
  uint64_t m = n - 1;
  for (uint64_t p = 2; p * p <= m; ++p) {
    if (m % p == 0) {
      fac.push_back(p);
      while (m % p == 0) m /= p;
    }
  }
  if (m > 1) fac.push_back(m);
  for (uint64_t w = 2; w < n; ++w) {
    bool ok = true;
    for (uint64_t q : fac)
      if (powmod(w, (n - 1) / q, n) == 1) {
        ok = false;
        break;
      }
    if (ok) return w;
  }
  return 0;
}

static inline double bern2(double t) { return t * t - t + 1.0 / 6.0; }

constexpr int kRerank = 32;

// T(z) with Neumaier summation in ascending k (one candidate per thread).
static double candidate_sum(uint64_t n, const std::vector<double>& p, uint64_t z) {
  double s = 0.0, c = 0.0;
  uint64_t r = 0;
  for (uint64_t k = 0; k < n; ++k) {
    double v = p[k] * bern2((double)r / (double)n);
    double t = s + v;
    if (std::fabs(s) >= std::fabs(v)) c += (s - t) + v;
    else c += (v - t) + s;
    s = t;
    r += z;
    if (r >= n) r -= n;
  }
  return s + c;
}




static uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// max_k 4^k e^2_k for the vector so far (products p over the N points)
// extended by component z with weight gamma.
static double embedded_criterion(const std::vector<double>& p, int K, int kmin, uint64_t z, double gamma) {
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

constexpr int kRerankEmb = 16;

// The criterion max_k 4^k e^2_k of every candidate z = 5^b mod N (b < N/4,
// reported as min(z, N - z)), from the per-v cyclic correlations.
static void embedded_all(const std::vector<double>& p, int K, int kmin, double gamma, std::vector<uint64_t>& zs,
                         std::vector<double>& crit) {
  const uint64_t N = 1ull << K;
  const uint64_t L0 = N / 4;
  zs.resize(L0);
  crit.assign(L0, 0.0);
  // level sums S_v(b), accumulated into per-k partial sums below
  std::vector<std::vector<double>> T(K);
  for (int v = 0; v < K; ++v) {
    const uint64_t Nv = N >> v;
    if (Nv < 8) continue;  // small groups: direct sums below
    const uint64_t L = Nv / 4;
    int logL = 0;
    while ((1ull << logL) < L) ++logL;
    std::vector<cd> q(L), w(L);
    uint64_t pw = 1;  // 5^a mod Nv
    for (uint64_t a = 0; a < L; ++a) {
      q[a] = cd(p[(pw << v)] + p[((Nv - pw) << v)], 0.0);
      w[a] = cd(1.0 + gamma * bern2((double)pw / (double)Nv), 0.0);
      pw = (pw * 5) & (Nv - 1);
    }
    std::vector<cd> tw(std::max<uint64_t>(1, L / 2));
    for (uint64_t k = 0; k < L / 2; ++k) tw[k] = std::polar(1.0, -2.0 * M_PI * (double)k / (double)L);
    fft(q, tw, logL, false);
    fft(w, tw, logL, false);
    for (uint64_t f = 0; f < L; ++f) q[f] = std::conj(q[f]) * w[f];
    fft(q, tw, logL, true);
    T[v].resize(L);
    for (uint64_t b = 0; b < L; ++b) T[v][b] = q[b].real() / (double)L;
  }
  parallel_for(L0, [&](size_t lo, size_t hi) {
    std::vector<double> lv(K + 1);
    uint64_t z = 1;  // 5^lo mod N
    {
      uint64_t base = 5, e = lo;
      while (e) {
        if (e & 1) z = (z * base) & (N - 1);
        base = (base * base) & (N - 1);
        e >>= 1;
      }
    }
    for (size_t b = lo; b < hi; ++b) {
      // contribution of the points with v trailing zero bits; J = 0 in every level
      for (int v = 0; v < K; ++v) {
        const uint64_t Nv = N >> v;
        double s;
        if (Nv >= 8) {
          s = T[v][b & (Nv / 4 - 1)];
        } else {
          s = 0.0;
          for (uint64_t u = 1; u < Nv; u += 2)
            s += p[u << v] * (1.0 + gamma * bern2((double)((u * z) & (Nv - 1)) / (double)Nv));
        }
        lv[v] = s;
      }
      double level_sum = p[0] * (1.0 + gamma * bern2(0.0)), worst = -1e300;
      for (int k = 0; k <= K; ++k) {  // size 2^k holds the points with v >= K - k
        if (k > 0) level_sum += lv[K - k];
        if (k < kmin) continue;
        worst = std::max(worst, std::ldexp(level_sum / (double)(1ull << k) - 1.0, 2 * k));
      }
      crit[b] = worst;
      zs[b] = std::min(z, N - z);
      z = (z * 5) & (N - 1);
    }
  });
}

}  // namespace qmc

using namespace qmc;

extern "C" int qmc_make_lattice(int32_t d, uint64_t n, const double* gamma, uint64_t* g_out) {
  if (d < 1 || d > QMC_DMAX) return fail(QMC_EINVAL, "d=%d outside [1, %d]", d, QMC_DMAX);
  if (!gamma || !g_out) return fail(QMC_EINVAL, "null gamma or g_out");
  if (n < 5 || n >= (1ull << 31) || !prime_check(n))
    return fail(QMC_EINVAL, "n=%llu must be a prime in [5, 2^31)", (unsigned long long)n);
  for (int i = 0; i < d; ++i)
    if (!(gamma[i] > 0.0) || !std::isfinite(gamma[i])) return fail(QMC_EINVAL, "gamma[%d] must be > 0", i);
  try {
    g_out[0] = 1;
    std::vector<double> p(n);
    parallel_for(n, [&](size_t lo, size_t hi) {
      for (size_t k = lo; k < hi; ++k) p[k] = 1.0 + gamma[0] * bern2((double)k / (double)n);
    });
    if (d == 1) return QMC_OK;
    const uint64_t w = primitive_root(n);
    const uint64_t h = (n - 1) / 2;
    std::vector<uint32_t> perm(n - 1);
    {
      uint64_t v = 1;
      for (uint64_t t = 0; t < n - 1; ++t) {
        perm[t] = (uint32_t)v;
        v = v * w % n;
      }
    }
    int logM = 0;
    while (((uint64_t)1 << logM) < 2 * h - 1) ++logM;
    const size_t M = (size_t)1 << logM;
    std::vector<cd> tw(M / 2);
    parallel_for(M / 2, [&](size_t lo, size_t hi) {
      for (size_t k = lo; k < hi; ++k) {
        double ang = -2.0 * M_PI * (double)k / (double)M;
        tw[k] = cd(std::cos(ang), std::sin(ang));
      }
    });
    std::vector<cd> chat(M, cd(0.0, 0.0));
    for (uint64_t t = 0; t < h; ++t) chat[t] = cd(bern2((double)perm[t] / (double)n), 0.0);
    fft(chat, tw, logM, false);
    std::vector<cd> work(M);
    std::vector<double> T(h);
    for (int s = 1; s < d; ++s) {
      // q[b] = p[w^(-b)], folded: q'[b] = q[b] + q[b + h]
      std::fill(work.begin(), work.end(), cd(0.0, 0.0));
      parallel_for(h, [&](size_t lo, size_t hi) {
        for (size_t b = lo; b < hi; ++b) {
          size_t nb1 = b == 0 ? 0 : (n - 1) - b;
          size_t nb2 = (n - 1) - (b + h);
          work[b] = cd(p[perm[nb1]] + p[perm[nb2]], 0.0);
        }
      });
      fft(work, tw, logM, false);
      parallel_for(M, [&](size_t lo, size_t hi) {
        for (size_t i = lo; i < hi; ++i) work[i] *= chat[i];
      });
      fft(work, tw, logM, true);
      const double inv = 1.0 / (double)M;
      for (uint64_t a = 0; a < h; ++a) {
        double v = work[a].real();
        if (a + h < M) v += work[a + h].real();
        T[a] = v * inv;
      }
      // exact re-ranking of the FFT's best candidates
      const uint64_t K = std::min<uint64_t>(kRerank, h);
      std::vector<uint64_t> order(h);
      for (uint64_t a = 0; a < h; ++a) order[a] = a;
      std::nth_element(order.begin(), order.begin() + (K - 1), order.end(),
                       [&](uint64_t x, uint64_t y) { return T[x] < T[y]; });
      std::vector<uint64_t> cz;
      for (uint64_t q = 0; q < K; ++q) cz.push_back(std::min<uint64_t>(perm[order[q]], n - perm[order[q]]));
      std::sort(cz.begin(), cz.end());
      cz.erase(std::unique(cz.begin(), cz.end()), cz.end());
      std::vector<double> exact(cz.size());
      {
        std::vector<std::thread> th;
        for (size_t q = 0; q < cz.size(); ++q)
          th.emplace_back([&, q] { exact[q] = candidate_sum(n, p, cz[q]); });
        for (auto& x : th) x.join();
      }
      uint64_t z = cz[0];
      double bestv = exact[0];
      for (size_t q = 1; q < cz.size(); ++q)
        if (exact[q] < bestv) {
          bestv = exact[q];
          z = cz[q];
        }
      g_out[s] = z;
      const double gs = gamma[s];
      parallel_for(n, [&](size_t lo, size_t hi) {
        for (size_t k = lo; k < hi; ++k) p[k] *= 1.0 + gs * bern2((double)mulmod(k, z, n) / (double)n);
      });
    }
  } catch (const std::bad_alloc&) {
    return fail(QMC_ENOMEM, "host memory for the CBC search");
  }
  return QMC_OK;
}

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
//
// All candidates at once.  Write J = 2^v u with u odd.  Modulo N_v = N / 2^v
// the odd residues are +-5^a (a < L_v = N_v / 4) and B2 is symmetric, so for
// z = +-5^b the points with that v contribute
//   T_v(b) = sum_a q_v[a] w_v[(a + b) mod L_v],
//   q_v[a] = p[2^v 5^a] + p[2^v (N_v - 5^a)],  w_v[c] = 1 + gamma B2(5^c mod N_v / N_v),
// a cyclic correlation of length L_v done by FFT.  Every embedded size 2^k
// uses the same T_v (those with v >= K - k), so one set of correlations per
// component gives every candidate's criterion in O(N log N); the kRerankEmb
// best are then recomputed exactly (term by term) and the smallest wins.

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
    if ((uint64_t)candidates >= odd_count && K >= 5) {
      // every odd candidate, by the correlations; the best few re-ranked exactly
      std::vector<uint64_t> zs;
      std::vector<double> cr;
      embedded_all(p, K, log2_nmin, gamma[s], zs, cr);
      std::vector<size_t> order(zs.size());
      for (size_t q = 0; q < order.size(); ++q) order[q] = q;
      const size_t top = std::min<size_t>(kRerankEmb, order.size());
      std::partial_sort(order.begin(), order.begin() + top, order.end(), [&](size_t x, size_t y) {
        return cr[x] < cr[y] || (cr[x] == cr[y] && zs[x] < zs[y]);
      });
      for (size_t q = 0; q < top; ++q) cand.push_back(zs[order[q]]);
      std::sort(cand.begin(), cand.end());
      cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    } else if ((uint64_t)candidates >= odd_count) {
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

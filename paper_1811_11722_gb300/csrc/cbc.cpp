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

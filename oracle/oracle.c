/*
 * Plain FP64 CPU oracle for the randomly shifted rank-1 lattice rule.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product links, loads or calls this
 * file; only the tests, the smoke check and the benchmark's CPU-baseline leg
 * do.  It shares no code, header or table with the CUDA path.
 *
 * Everything here is the paper's definition written out, point by point, in
 * double precision, with no blocking or reordering beyond the definition:
 *   Eq. (2)  x_{j,k} = {(j-1) g / n + Delta_k},  Q^(k) = (1/n) sum_j f(x_{j,k}),
 *            Qbar = (1/m) sum_k Q^(k)
 *   Eq. (3)  sigma^2 = 1/(m(m-1)) sum_k (Q^(k) - Qbar)^2, real and imaginary
 *            parts estimated separately
 *   Eq. (5)  Korobov transform of weight alpha: z = int_0^x w, w(u) =
 *            u^a (1-u)^a / B(a+1, a+1); the rule integrates f(z(x)) prod_i w(x_i)
 *   Eq. (6)  baker's transform z = 1 - |2x - 1| (weight 1)
 *   Eq. (7)  integrand class prod_j P_j^{a_j + b_j eps}: here U^{aU} F^{aF} at
 *            eps = 0, and the coefficient integrands of its eps expansion,
 *            U^{aU} F^{aF} (bU log U + bF log F)^k / k!
 *   Sec. 3   contour deformation z_k = y_k - i lambda y_k (1 - y_k) dF/dy_k,
 *            which vanishes at the endpoints y_k in {0, 1}
 * Per-shift sums use Neumaier's compensated summation.  Threads, when asked
 * for, split j into fixed contiguous chunks whose sums are combined in chunk
 * order, so the result does not depend on scheduling.
 *
 * Generating-vector search (not in the paper; the paper takes g as given):
 * component-by-component (CBC) minimisation of the shift-averaged worst-case
 * error in the unanchored weighted Sobolev space with product weights,
 *   e^2(g) = -1 + (1/n) sum_{k=0}^{n-1} prod_i (1 + gamma_i B2({k g_i / n})),
 *   B2(t) = t^2 - t + 1/6,
 * plain O(n^2) per dimension, g_1 = 1, candidates 1 <= z <= (n-1)/2, ties to
 * the smallest z.  The candidate criterion T(z) = sum_k p[k] B2({k z/n}) is
 * also what the FFT-based search (cbc.py) re-ranks its best candidates by.
 */
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_DMAX 64

enum { ORC_CONST = 0, ORC_SEPARABLE_EXP = 1, ORC_SECTOR = 2, ORC_SECTOR_DEFORMED = 3, ORC_TRIG = 4 };
enum { ORC_T_NONE = 0, ORC_T_KOROBOV = 1, ORC_T_BAKER = 2 };

typedef struct {
  int kind;
  int d;
  int tkind;
  int alpha;
  int nU;
  const double* cU;      /* nU coefficients */
  const uint8_t* eU;     /* nU x d exponents, row-major */
  int nF;
  const double* cF;
  const uint8_t* eF;
  int aU, aF;            /* integer powers (eps = 0) */
  double lambda;         /* deformation parameter */
  const double* c;       /* separable: prod (1 + c_i z_i) exp(b_i z_i) */
  const double* b;
  const int32_t* h;      /* trig: cos(2 pi h . z) */
  /* optional control variate g(z) = sum_{r<cvR} prod_{i<d} sum_{k<cvK}
   * a[(r*d + i)*cvK + k] cos(cvF pi k z_i), subtracted from f at the
   * transformed point z (so the value becomes (f - g)(z) prod_i w_i) */
  int cvR, cvK, cvF;
  const float* cva;
  /* epsilon expansion of Eq. (7): U^(aU + bU eps) F^(aF + bF eps) =
   * sum_k eps^k U^aU F^aF (bU log U + bF log F)^k / k!; eps_order = k selects
   * the coefficient integrand (0 = the plain U^aU F^aF) */
  int eps_order;
  double eps_bU, eps_bF;
} orc_problem;

/* ---------------------------------------------------------------- sums --- */

typedef struct {
  double s, c;
} neum_t;

static void neum_add(neum_t* a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v))
    a->c += (a->s - t) + v;
  else
    a->c += (v - t) + a->s;
  a->s = t;
}

static double neum_get(const neum_t* a) { return a->s + a->c; }

/* ----------------------------------------------------------- transforms --- */

/* Beta(alpha+1, alpha+1)^-1 = (2 alpha + 1)! / (alpha!)^2 */
static double korobov_norm(int alpha) {
  double num = 1.0, den = 1.0;
  for (int i = 1; i <= 2 * alpha + 1; ++i) num *= (double)i;
  for (int i = 1; i <= alpha; ++i) den *= (double)i;
  return num / (den * den);
}

static double binom(int a, int k) {
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (double)(a - k + i) / (double)i;
  return r;
}

/* z(x) = int_0^x u^a (1-u)^a du / B for x <= 1/2, expanding (1-u)^a by the
 * binomial theorem and integrating term by term. */
static double korobov_z_lower(int alpha, double x) {
  double s = 0.0;
  for (int k = 0; k <= alpha; ++k) {
    double term = binom(alpha, k) * pow(x, (double)(alpha + k + 1)) / (double)(alpha + k + 1);
    s += (k & 1) ? -term : term;
  }
  return s * korobov_norm(alpha);
}

/* Eq. (5) and (6).  Returns z; *w receives the Jacobian weight. */
double orc_transform(int tkind, int alpha, double x, double* w) {
  if (tkind == ORC_T_KOROBOV) {
    *w = korobov_norm(alpha) * pow(x, (double)alpha) * pow(1.0 - x, (double)alpha);
    /* w is symmetric about 1/2, so z(x) = 1 - z(1 - x) */
    if (x <= 0.5) return korobov_z_lower(alpha, x);
    return 1.0 - korobov_z_lower(alpha, 1.0 - x);
  }
  if (tkind == ORC_T_BAKER) {
    *w = 1.0;
    return 1.0 - fabs(2.0 * x - 1.0);
  }
  *w = 1.0;
  return x;
}

/* ----------------------------------------------------------- polynomials --- */

static double poly_eval_real(int nt, const double* c, const uint8_t* e, int d, const double* y) {
  double s = 0.0;
  for (int t = 0; t < nt; ++t) {
    double p = c[t];
    for (int i = 0; i < d; ++i)
      for (int q = 0; q < e[t * d + i]; ++q) p *= y[i];
    s += p;
  }
  return s;
}

static double complex poly_eval_cplx(int nt, const double* c, const uint8_t* e, int d,
                                     const double complex* z) {
  double complex s = 0.0;
  for (int t = 0; t < nt; ++t) {
    double complex p = c[t];
    for (int i = 0; i < d; ++i)
      for (int q = 0; q < e[t * d + i]; ++q) p *= z[i];
    s += p;
  }
  return s;
}

/* d/dy_k of the polynomial at y (monomial rule: e_k y_k^(e_k - 1) prod_{i != k} y_i^e_i) */
static double poly_deriv1(int nt, const double* c, const uint8_t* e, int d, const double* y, int k) {
  double s = 0.0;
  for (int t = 0; t < nt; ++t) {
    int ek = e[t * d + k];
    if (ek == 0) continue;
    double p = c[t] * (double)ek;
    for (int i = 0; i < d; ++i) {
      int ei = e[t * d + i] - (i == k ? 1 : 0);
      for (int q = 0; q < ei; ++q) p *= y[i];
    }
    s += p;
  }
  return s;
}

/* d^2/(dy_k dy_l) of the polynomial at y */
static double poly_deriv2(int nt, const double* c, const uint8_t* e, int d, const double* y, int k, int l) {
  double s = 0.0;
  for (int t = 0; t < nt; ++t) {
    int ek = e[t * d + k];
    int el = e[t * d + l];
    double p;
    if (k == l) {
      if (ek < 2) continue;
      p = c[t] * (double)ek * (double)(ek - 1);
    } else {
      if (ek == 0 || el == 0) continue;
      p = c[t] * (double)ek * (double)el;
    }
    for (int i = 0; i < d; ++i) {
      int ei = e[t * d + i] - (i == k ? 1 : 0) - (i == l ? 1 : 0);
      for (int q = 0; q < ei; ++q) p *= y[i];
    }
    s += p;
  }
  return s;
}

static double complex cpow_int(double complex z, int a) {
  double complex r = 1.0;
  int k = a < 0 ? -a : a;
  for (int i = 0; i < k; ++i) r *= z;
  return a < 0 ? 1.0 / r : r;
}

static double pow_int(double x, int a) {
  double r = 1.0;
  int k = a < 0 ? -a : a;
  for (int i = 0; i < k; ++i) r *= x;
  return a < 0 ? 1.0 / r : r;
}

/* Determinant by LU factorisation with partial pivoting (row swaps flip sign). */
double complex orc_det_lu(int d, double complex* a /* d x d, destroyed */) {
  double complex det = 1.0;
  for (int c = 0; c < d; ++c) {
    int piv = c;
    double best = cabs(a[c * d + c]);
    for (int r = c + 1; r < d; ++r) {
      double v = cabs(a[r * d + c]);
      if (v > best) {
        best = v;
        piv = r;
      }
    }
    if (best == 0.0) return 0.0;
    if (piv != c) {
      for (int q = 0; q < d; ++q) {
        double complex t = a[c * d + q];
        a[c * d + q] = a[piv * d + q];
        a[piv * d + q] = t;
      }
      det = -det;
    }
    det *= a[c * d + c];
    for (int r = c + 1; r < d; ++r) {
      double complex f = a[r * d + c] / a[c * d + c];
      for (int q = c; q < d; ++q) a[r * d + q] -= f * a[c * d + q];
    }
  }
  return det;
}

/* ctypes cannot take a complex return value: write (re, im) to out. */
void orc_det_lu_out(int d, double complex* a, double* out) {
  double complex r = orc_det_lu(d, a);
  out[0] = creal(r);
  out[1] = cimag(r);
}

/* ------------------------------------------------------------- integrand --- */

/* f at the (already transformed) point y.  out[0] = Re, out[1] = Im.
 * *bad is set when the deformed F has a positive imaginary part (the wrong
 * side of the Feynman prescription). */
int orc_integrand(const orc_problem* p, const double* y, double* out, int* bad) {
  int d = p->d;
  *bad = 0;
  out[1] = 0.0;
  switch (p->kind) {
    case ORC_CONST:
      out[0] = 1.0;
      return 0;
    case ORC_SEPARABLE_EXP: {
      double v = 1.0;
      for (int i = 0; i < d; ++i) v *= (1.0 + p->c[i] * y[i]) * exp(p->b[i] * y[i]);
      out[0] = v;
      return 0;
    }
    case ORC_TRIG: {
      double ph = 0.0;
      for (int i = 0; i < d; ++i) ph += (double)p->h[i] * y[i];
      out[0] = cos(2.0 * M_PI * ph);
      return 0;
    }
    case ORC_SECTOR: {
      double U = poly_eval_real(p->nU, p->cU, p->eU, d, y);
      double F = poly_eval_real(p->nF, p->cF, p->eF, d, y);
      out[0] = pow_int(U, p->aU) * pow_int(F, p->aF);
      if (p->eps_order > 0) {
        double L = p->eps_bU * log(U) + p->eps_bF * log(F);
        double c = 1.0;
        for (int k = 1; k <= p->eps_order; ++k) c *= L / (double)k;
        out[0] *= c;
      }
      return 0;
    }
    case ORC_SECTOR_DEFORMED: {
      double grad[ORC_DMAX];
      double complex z[ORC_DMAX];
      double complex J[ORC_DMAX * ORC_DMAX];
      double lam = p->lambda;
      for (int k = 0; k < d; ++k) grad[k] = poly_deriv1(p->nF, p->cF, p->eF, d, y, k);
      for (int k = 0; k < d; ++k) z[k] = y[k] - I * lam * y[k] * (1.0 - y[k]) * grad[k];
      /* J_kl = dz_k/dy_l = delta_kl - i lam [delta_kl (1 - 2 y_k) dF_k + y_k (1 - y_k) d2F_kl] */
      for (int k = 0; k < d; ++k)
        for (int l = 0; l < d; ++l) {
          double h2 = poly_deriv2(p->nF, p->cF, p->eF, d, y, k, l);
          double re = (k == l) ? 1.0 : 0.0;
          double im = -lam * (((k == l) ? (1.0 - 2.0 * y[k]) * grad[k] : 0.0) + y[k] * (1.0 - y[k]) * h2);
          J[k * d + l] = re + I * im;
        }
      double complex detJ = orc_det_lu(d, J);
      double complex U = poly_eval_cplx(p->nU, p->cU, p->eU, d, z);
      double complex F = poly_eval_cplx(p->nF, p->cF, p->eF, d, z);
      if (cimag(F) > 0.0) *bad = 1;
      double complex v = cpow_int(U, p->aU) * cpow_int(F, p->aF) * detJ;
      out[0] = creal(v);
      out[1] = cimag(v);
      return 0;
    }
  }
  return -1;
}

/* ------------------------------------------------------- control variate --- */

/* g(x) = sum_r prod_i sum_k a_rik cos(F pi k x_i), each cosine from libm. */
double orc_cv_g(int d, int R, int K, int F, const float* a, const double* x) {
  double g = 0.0;
  for (int r = 0; r < R; ++r) {
    double prod = 1.0;
    for (int i = 0; i < d; ++i) {
      double s = 0.0;
      for (int k = 0; k < K; ++k) s += (double)a[(r * d + i) * K + k] * cos((double)F * M_PI * (double)k * x[i]);
      prod *= s;
    }
    g += prod;
  }
  return g;
}

/* int_[0,1]^d g = sum_r prod_i a_ri0, since int_0^1 cos(F pi k x) dx = 0 for k >= 1. */
double orc_cv_integral(int d, int R, int K, const float* a) {
  double s = 0.0;
  for (int r = 0; r < R; ++r) {
    double p = 1.0;
    for (int i = 0; i < d; ++i) p *= (double)a[(r * d + i) * K];
    s += p;
  }
  return s;
}

/* Mean squared error L = (1/P) sum_j (g(x_j) - h_j)^2 and its gradient
 * dL/da_rik = (2/P) sum_j (g_j - h_j) prod_{i' != i} C_ri'(x_j) cos(F pi k x_ji),
 * C_ri(x) = sum_k a_rik cos(F pi k x_i), in FP64 (chain rule, term by term). */
double orc_cv_loss_grad(int d, int R, int K, int F, int P, const double* x, const double* h, const float* a,
                        double* grad) {
  int na = R * d * K;
  for (int q = 0; q < na; ++q) grad[q] = 0.0;
  double* C = (double*)malloc(sizeof(double) * R * d);
  double* cs = (double*)malloc(sizeof(double) * d * K);
  neum_t loss = {0, 0};
  for (int j = 0; j < P; ++j) {
    const double* xj = x + (size_t)j * d;
    for (int i = 0; i < d; ++i)
      for (int k = 0; k < K; ++k) cs[i * K + k] = cos((double)F * M_PI * (double)k * xj[i]);
    double g = 0.0;
    for (int r = 0; r < R; ++r) {
      double prod = 1.0;
      for (int i = 0; i < d; ++i) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += (double)a[(r * d + i) * K + k] * cs[i * K + k];
        C[r * d + i] = s;
        prod *= s;
      }
      g += prod;
    }
    double e = g - h[j];
    neum_add(&loss, e * e);
    for (int r = 0; r < R; ++r)
      for (int i = 0; i < d; ++i) {
        double other = 1.0;
        for (int i2 = 0; i2 < d; ++i2)
          if (i2 != i) other *= C[r * d + i2];
        for (int k = 0; k < K; ++k) grad[(r * d + i) * K + k] += 2.0 * e * other * cs[i * K + k] / (double)P;
      }
  }
  free(C);
  free(cs);
  return neum_get(&loss) / (double)P;
}

/* The fit's contractions on BF16 operands (the configuration's "BF16
 * inputs, FP32 accumulate" for training the surrogate): the same loss and
 * gradient as orc_cv_loss_grad, with every operand of the two contractions
 * rounded first to float and then to bfloat16 (round to nearest, ties to
 * even) -- the basis values cos(F pi k x), the parameters a, and the factor
 * 2 e prod_{i' != i} C_ri' / P of the gradient -- and their exact products
 * summed in FP64. */
double orc_bf16(double v) {
  float f = (float)v;
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7F800000u) == 0x7F800000u) return (double)f; /* Inf / NaN kept */
  u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
  memcpy(&f, &u, 4);
  return (double)f;
}

double orc_cv_loss_grad_bf16(int d, int R, int K, int F, int P, const double* x, const double* h, const float* a,
                             double* grad) {
  int na = R * d * K;
  for (int q = 0; q < na; ++q) grad[q] = 0.0;
  double* C = (double*)malloc(sizeof(double) * R * d);
  double* cs = (double*)malloc(sizeof(double) * d * K);
  double* ab = (double*)malloc(sizeof(double) * na);
  for (int q = 0; q < na; ++q) ab[q] = orc_bf16((double)a[q]);
  neum_t loss = {0, 0};
  for (int j = 0; j < P; ++j) {
    const double* xj = x + (size_t)j * d;
    for (int i = 0; i < d; ++i)
      for (int k = 0; k < K; ++k) cs[i * K + k] = orc_bf16(cos((double)F * M_PI * (double)k * xj[i]));
    double g = 0.0;
    for (int r = 0; r < R; ++r) {
      double prod = 1.0;
      for (int i = 0; i < d; ++i) {
        double s = 0.0;
        for (int k = 0; k < K; ++k) s += ab[(r * d + i) * K + k] * cs[i * K + k];
        C[r * d + i] = s;
        prod *= s;
      }
      g += prod;
    }
    double e = g - h[j];
    neum_add(&loss, e * e);
    for (int r = 0; r < R; ++r)
      for (int i = 0; i < d; ++i) {
        double other = 1.0;
        for (int i2 = 0; i2 < d; ++i2)
          if (i2 != i) other *= C[r * d + i2];
        const double dg = orc_bf16(2.0 * e * other / (double)P);
        for (int k = 0; k < K; ++k) grad[(r * d + i) * K + k] += dg * cs[i * K + k];
      }
  }
  free(C);
  free(cs);
  free(ab);
  return neum_get(&loss) / (double)P;
}

/* ------------------------------------------------------------- the rule --- */

/* Lattice index of Eq. (2): idx_i = ((j-1) g_i) mod n with j-1 = jm1, exact in 128 bits. */
uint64_t orc_index(uint64_t jm1, uint64_t g, uint64_t n) {
  return (uint64_t)(((unsigned __int128)jm1 * (unsigned __int128)g) % (unsigned __int128)n);
}

/* One point: x_i = {idx_i / n + Delta_i}; z_i, w_i from the transform;
 * value = f(z) prod_i w_i.  Optional dumps of idx, x, z. */
int orc_point(const orc_problem* p, uint64_t n, const uint64_t* g, const double* shift, uint64_t jm1,
              double* val, uint64_t* idx_out, double* x_out, double* z_out, int* bad) {
  double x[ORC_DMAX], z[ORC_DMAX];
  double wprod = 1.0;
  for (int i = 0; i < p->d; ++i) {
    uint64_t idx = orc_index(jm1, g[i], n);
    double y = (double)idx / (double)n + shift[i];
    x[i] = (y >= 1.0) ? y - 1.0 : y;
    double w;
    z[i] = orc_transform(p->tkind, p->alpha, x[i], &w);
    wprod *= w;
    if (idx_out) idx_out[i] = idx;
    if (x_out) x_out[i] = x[i];
    if (z_out) z_out[i] = z[i];
  }
  double f[2];
  orc_integrand(p, z, f, bad);
  val[0] = f[0] * wprod;
  val[1] = f[1] * wprod;
  if (p->cva) {
    /* Q[f - g] + int g: the surrogate is subtracted from f before the
     * transform, so the rule sums (f - g)(z(x)) prod_i w(x_i) */
    val[0] -= orc_cv_g(p->d, p->cvR, p->cvK, p->cvF, p->cva, z) * wprod;
  }
  return 0;
}

typedef struct {
  const orc_problem* p;
  uint64_t n;
  const uint64_t* g;
  int m;
  const double* shifts;
  uint64_t j0, j1;
  neum_t* acc;        /* m x 2 */
  uint64_t* nonfinite; /* m */
  uint64_t bad;
} orc_chunk;

static void* orc_chunk_run(void* arg) {
  orc_chunk* c = (orc_chunk*)arg;
  const orc_problem* p = c->p;
  for (int k = 0; k < c->m; ++k) {
    const double* sh = c->shifts + (size_t)k * p->d;
    for (uint64_t j = c->j0; j < c->j1; ++j) {
      double v[2];
      int bad = 0;
      orc_point(p, c->n, c->g, sh, j, v, NULL, NULL, NULL, &bad);
      c->bad += (uint64_t)bad;
      if (!isfinite(v[0]) || !isfinite(v[1])) {
        c->nonfinite[k] += 1;
        continue;
      }
      neum_add(&c->acc[2 * k + 0], v[0]);
      neum_add(&c->acc[2 * k + 1], v[1]);
    }
  }
  return NULL;
}

/* Per-shift sums S_k = sum_{j in [j0, j1)} f(x_{j,k}) (re, im), with 0-based j
 * standing for the paper's j-1.  Non-finite values are counted per shift and
 * left out of the sum.  nthreads >= 1 splits [j0, j1) into that many fixed
 * contiguous chunks. */
int orc_rule_sums(const orc_problem* p, uint64_t n, const uint64_t* g, int m, const double* shifts,
                  uint64_t j0, uint64_t j1, int nthreads, double* sums, uint64_t* nonfinite,
                  uint64_t* deform_bad) {
  if (nthreads < 1) nthreads = 1;
  if (p->d < 1 || p->d > ORC_DMAX || j1 < j0) return -1;
  orc_chunk* ch = (orc_chunk*)calloc((size_t)nthreads, sizeof(orc_chunk));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  uint64_t len = j1 - j0;
  for (int t = 0; t < nthreads; ++t) {
    ch[t].p = p;
    ch[t].n = n;
    ch[t].g = g;
    ch[t].m = m;
    ch[t].shifts = shifts;
    ch[t].j0 = j0 + len * (uint64_t)t / (uint64_t)nthreads;
    ch[t].j1 = j0 + len * (uint64_t)(t + 1) / (uint64_t)nthreads;
    ch[t].acc = (neum_t*)calloc((size_t)m * 2, sizeof(neum_t));
    ch[t].nonfinite = (uint64_t*)calloc((size_t)m, sizeof(uint64_t));
  }
  if (nthreads == 1) {
    orc_chunk_run(&ch[0]);
  } else {
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, orc_chunk_run, &ch[t]);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  }
  uint64_t bad = 0;
  for (int k = 0; k < m; ++k) {
    neum_t re = {0, 0}, im = {0, 0};
    uint64_t nf = 0;
    for (int t = 0; t < nthreads; ++t) {
      neum_add(&re, neum_get(&ch[t].acc[2 * k]));
      neum_add(&im, neum_get(&ch[t].acc[2 * k + 1]));
      nf += ch[t].nonfinite[k];
    }
    sums[2 * k] = neum_get(&re);
    sums[2 * k + 1] = neum_get(&im);
    if (nonfinite) nonfinite[k] = nf;
  }
  for (int t = 0; t < nthreads; ++t) {
    bad += ch[t].bad;
    free(ch[t].acc);
    free(ch[t].nonfinite);
  }
  if (deform_bad) *deform_bad = bad;
  free(ch);
  free(th);
  return 0;
}

/* Eq. (2) and (3) from per-shift sums: Q^(k) = S_k / n, Qbar, sigma^2 (two-pass),
 * separately for the real and the imaginary part. */
int orc_estimate(int m, uint64_t n, const double* sums, double* q, double* mean, double* var) {
  if (m < 2) return -1;
  for (int part = 0; part < 2; ++part) {
    neum_t s = {0, 0};
    for (int k = 0; k < m; ++k) {
      q[2 * k + part] = sums[2 * k + part] / (double)n;
      neum_add(&s, q[2 * k + part]);
    }
    double qbar = neum_get(&s) / (double)m;
    neum_t v = {0, 0};
    for (int k = 0; k < m; ++k) {
      double dlt = q[2 * k + part] - qbar;
      neum_add(&v, dlt * dlt);
    }
    mean[part] = qbar;
    var[part] = neum_get(&v) / ((double)m * (double)(m - 1));
  }
  return 0;
}

/* ------------------------------------------------- Gauss-Legendre check --- */

typedef struct {
  const orc_problem* p;
  int q;
  const double* nodes;   /* on [0, 1] */
  const double* weights; /* on [0, 1] */
  uint64_t i0, i1;
  neum_t acc[2];
} orc_gl_chunk;

static void* orc_gl_run(void* arg) {
  orc_gl_chunk* c = (orc_gl_chunk*)arg;
  int d = c->p->d;
  double y[ORC_DMAX];
  for (uint64_t t = c->i0; t < c->i1; ++t) {
    uint64_t r = t;
    double w = 1.0;
    for (int i = 0; i < d; ++i) {
      int a = (int)(r % (uint64_t)c->q);
      r /= (uint64_t)c->q;
      y[i] = c->nodes[a];
      w *= c->weights[a];
    }
    double f[2];
    int bad;
    orc_integrand(c->p, y, f, &bad);
    neum_add(&c->acc[0], w * f[0]);
    neum_add(&c->acc[1], w * f[1]);
  }
  return NULL;
}

/* Tensor-product Gauss-Legendre integral of f over [0,1]^d (no transform). */
int orc_gauss_legendre(const orc_problem* p, int q, const double* nodes, const double* weights,
                       int nthreads, double* out) {
  uint64_t total = 1;
  for (int i = 0; i < p->d; ++i) total *= (uint64_t)q;
  if (nthreads < 1) nthreads = 1;
  orc_gl_chunk* ch = (orc_gl_chunk*)calloc((size_t)nthreads, sizeof(orc_gl_chunk));
  pthread_t* th = (pthread_t*)calloc((size_t)nthreads, sizeof(pthread_t));
  for (int t = 0; t < nthreads; ++t) {
    ch[t].p = p;
    ch[t].q = q;
    ch[t].nodes = nodes;
    ch[t].weights = weights;
    ch[t].i0 = total * (uint64_t)t / (uint64_t)nthreads;
    ch[t].i1 = total * (uint64_t)(t + 1) / (uint64_t)nthreads;
  }
  for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, orc_gl_run, &ch[t]);
  for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
  neum_t re = {0, 0}, im = {0, 0};
  for (int t = 0; t < nthreads; ++t) {
    neum_add(&re, neum_get(&ch[t].acc[0]));
    neum_add(&im, neum_get(&ch[t].acc[1]));
  }
  out[0] = neum_get(&re);
  out[1] = neum_get(&im);
  free(ch);
  free(th);
  return 0;
}

/* ------------------------------------------------------------------ CBC --- */

static double bern2(double t) { return t * t - t + 1.0 / 6.0; }

/* e^2(g) = -1 + (1/n) sum_{k=0}^{n-1} prod_i (1 + gamma_i B2({k g_i / n})),
 * summed as (1/n) sum_k [prod_i (1 + a_i) - 1] with the bracket built up as
 * t <- t + a_i (1 + t), which avoids cancelling against the -1 when e^2 is
 * far below double resolution of 1. */
double orc_cbc_error(int d, uint64_t n, const uint64_t* g, const double* gamma) {
  neum_t s = {0, 0};
  for (uint64_t k = 0; k < n; ++k) {
    double t = 0.0;
    for (int i = 0; i < d; ++i) {
      uint64_t r = orc_index(k, g[i], n);
      double a = gamma[i] * bern2((double)r / (double)n);
      t = t + a * (1.0 + t);
    }
    neum_add(&s, t);
  }
  return neum_get(&s) / (double)n;
}

/* The part of e^2 that depends on the next component z, given the running
 * products p[k] = prod_{i<s} (1 + gamma_i B2({k g_i / n})):
 *   T(z) = sum_{k=0}^{n-1} p[k] B2({k z / n})   (Neumaier, k ascending).
 * e^2 with z appended = -1 + (1/n) sum_k p[k] + (gamma_s / n) T(z), so the
 * search minimises T. */
double orc_cbc_candidate(uint64_t n, const double* p, uint64_t z) {
  neum_t s = {0, 0};
  for (uint64_t k = 0; k < n; ++k) neum_add(&s, p[k] * bern2((double)orc_index(k, z, n) / (double)n));
  return neum_get(&s);
}

/* Plain component-by-component construction: g_1 = 1, then for each next
 * dimension the candidate z in [1, (n-1)/2] minimising T(z) (equivalently
 * e^2) given the earlier components (strict <, ascending z: ties go to the
 * smallest z). */
int orc_cbc_plain(int d, uint64_t n, const double* gamma, uint64_t* g) {
  if (d < 1 || n < 2) return -1;
  double* prodk = (double*)malloc(sizeof(double) * n);
  g[0] = 1;
  for (uint64_t k = 0; k < n; ++k) prodk[k] = 1.0 + gamma[0] * bern2((double)orc_index(k, 1, n) / (double)n);
  for (int s = 1; s < d; ++s) {
    uint64_t best_z = 1;
    double best = INFINITY;
    uint64_t zmax = (n - 1) / 2;
    if (zmax < 1) zmax = 1;
    for (uint64_t z = 1; z <= zmax; ++z) {
      double t = orc_cbc_candidate(n, prodk, z);
      if (t < best) {
        best = t;
        best_z = z;
      }
    }
    g[s] = best_z;
    for (uint64_t k = 0; k < n; ++k)
      prodk[k] *= 1.0 + gamma[s] * bern2((double)orc_index(k, best_z, n) / (double)n);
  }
  free(prodk);
  return 0;
}

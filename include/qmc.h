/*
 * qmc.h - C ABI of the GB300 (sm_103a) randomly shifted rank-1 lattice rule.
 *
 * The library evaluates, on one GPU,
 *   Qbar = (1/m) sum_{k=1}^{m} Q^(k),  Q^(k) = (1/n) sum_{j=1}^{n} f({(j-1) g / n + Delta_k})
 * (Eq. 2 of "Numerical evaluation of multi-loop integrals", Sec. 2) and the
 * error estimate
 *   sigma^2 = 1/(m(m-1)) sum_k (Q^(k) - Qbar)^2
 * (Eq. 3), for integrands f of the sector-decomposed class of Eq. (7) after a
 * periodizing transform (Korobov, Eq. 5, or baker, Eq. 6).
 *
 * Conventions shared by every entry point:
 *   - Every function returns a qmc_status; QMC_OK is 0.  No exception or
 *     longjmp crosses the ABI.
 *   - Input arrays (g, shifts, polynomial tables, weights, c, b, h) are HOST
 *     memory owned by the caller; the library reads them during the call and
 *     keeps no pointer to them afterwards.
 *   - Result arrays (qmc_result, per_shift) may be host or device memory; the
 *     library tells them apart with cudaPointerGetAttributes.  When a result
 *     lives in host memory the call synchronises `stream`; when every result
 *     lives in device memory the call is asynchronous on `stream`.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream).  All device work of a call is ordered on it.
 *   - Complex results are reported as two real estimates (real part and
 *     imaginary part), each by Eq. (3); index [0] is the real part, [1] the
 *     imaginary part.  Real integrands report 0 for [1].
 */
#ifndef QMC_H
#define QMC_H

#ifndef __CUDACC_RTC__
#include <stdint.h>
#endif

#ifdef __cplusplus
extern "C" {
#endif

#define QMC_DMAX 16 /* largest supported dimension d */

typedef enum {
  QMC_OK = 0,
  QMC_EINVAL = -1,       /* an argument is out of range or inconsistent */
  QMC_ENOMEM = -2,       /* a device or host allocation failed */
  QMC_ECUDA = -3,        /* a CUDA runtime call failed (no GPU, launch error, ...) */
  QMC_ENONFINITE = -4,   /* some f values were NaN/Inf; they were left out and counted */
  QMC_ETIMEOUT = -5,     /* a bounded device wait ran out */
  QMC_EDEFORM = -6,      /* deformed F had Im F > 0 at some points (counted) */
  QMC_EUNSUPPORTED = -7  /* a valid request this build has no kernel for */
} qmc_status;

/* Periodizing transform applied to every coordinate before f.
 * KOROBOV (Eq. 5): z = int_0^x w(u) du with w(u) = u^a (1-u)^a / B(a+1, a+1),
 *   alpha = a in [1, 6]; the rule integrates f(z(x)) prod_i w(x_i).
 * BAKER (Eq. 6): z = 1 - |2x - 1|, weight 1.
 * NONE: z = x. */
enum { QMC_TRANSFORM_NONE = 0, QMC_TRANSFORM_KOROBOV = 1, QMC_TRANSFORM_BAKER = 2 };
typedef struct {
  int32_t kind;
  int32_t alpha;
} qmc_transform;

/* Polynomial in d variables as a term table:
 *   P(z) = sum_{t < nterms} coef[t] * prod_{i < d} z_i ^ expo[t * d + i].
 * Total degree at most 3.  Repeated monomials are summed. */
typedef struct {
  int32_t nterms;
  const double* coef; /* [nterms] */
  const uint8_t* expo; /* [nterms * d], row-major */
} qmc_poly;

/* Integrand families.
 * CONST          f = 1                                 (Sec. 2 / Fig. 3 study)
 * SEPARABLE_EXP  f = prod_i (1 + c_i z_i) exp(b_i z_i)  (closed-form test integrand)
 * SECTOR         f = U(z)^aU F(z)^aF                   (Eq. 7 at eps = 0)
 * SECTOR_DEFORMED f = U(w)^aU F(w)^aF det(dw/dz), with the contour
 *                w_k = z_k - i lambda z_k (1 - z_k) dF/dz_k (Sec. 3 Feynman
 *                prescription; vanishes at z_k in {0, 1}); F of degree <= 2.
 *                FP32EVAL with Korobov 3, U of degree 1, powers (-2, -1),
 *                d <= 5 and J diagonally dominant on the cube evaluates two
 *                shifts per instruction; QMC_DEFORMED_PACKED=0 in the
 *                environment keeps one shift per thread (same results to
 *                FP32 rounding)
 * TRIG           f = cos(2 pi h . z)                   (dual-lattice check) */
enum {
  QMC_F_CONST = 0,
  QMC_F_SEPARABLE_EXP = 1,
  QMC_F_SECTOR = 2,
  QMC_F_SECTOR_DEFORMED = 3,
  QMC_F_TRIG = 4
};

/* Arithmetic of the per-point evaluation.  Per-shift sums, Q^(k), Qbar and
 * sigma^2 are FP64 on the device in both modes.
 * FP64: coordinates, transform and f in double.
 * FP32EVAL: coordinates from 32-bit fixed point, transform and f in float,
 *   compensated float run sums promoted to double per thread.  Under the
 *   Korobov transform every value enters the compensated sum on its own (its
 *   values span many binades) and the sector kernels form the weight from the
 *   product of the factors with one compensated cube; at n ~ 1.7e7 the FP32
 *   and FP64 per-shift values then agree to ~1e-10 per dimension. */
enum { QMC_FP64 = 0, QMC_FP32EVAL = 1 };

typedef struct {
  int32_t kind;      /* QMC_F_* */
  int32_t d;         /* dimension, 1 <= d <= QMC_DMAX; must equal the rule's d */
  int32_t precision; /* QMC_FP64 or QMC_FP32EVAL */
  qmc_poly U, F;     /* SECTOR / SECTOR_DEFORMED */
  int32_t aU, aF;    /* integer powers in [-8, 8] */
  double lambda;     /* SECTOR_DEFORMED deformation parameter */
  const double* c;   /* SEPARABLE_EXP: [d] */
  const double* b;   /* SEPARABLE_EXP: [d] */
  const int32_t* h;  /* TRIG: [d] */
} qmc_integrand;

typedef struct {
  double mean[2]; /* Qbar (Eq. 2), real and imaginary part */
  double var[2];  /* sigma^2 (Eq. 3) */
  double err[2];  /* sqrt(var) */
  uint64_t nonfinite;         /* points whose f was NaN/Inf (left out of the sums) */
  uint64_t deform_violations; /* SECTOR_DEFORMED points with Im F(w) > 0 */
  int32_t status;             /* qmc_status of this problem */
  int32_t reserved;
} qmc_result;

/* Generating vector by component-by-component search (the paper takes g as
 * given, Eq. 2; the construction follows the review it cites for QMC):
 * minimises, one component at a time with g_1 = 1, the shift-averaged
 * worst-case error in the unanchored weighted Sobolev space with product
 * weights,
 *   e^2(g) = -1 + (1/n) sum_{k=0}^{n-1} prod_i (1 + gamma_i B2({k g_i / n})),
 *   B2(t) = t^2 - t + 1/6,
 * over candidates 1 <= z <= (n-1)/2 (ties to the smallest z).
 *   d      1 <= d <= QMC_DMAX
 *   n      prime, 5 <= n < 2^31
 *   gamma  [d] positive weights (host)
 *   g_out  [d] result (host)
 * Host precompute: runs on the host cores (FFT-based cyclic convolution,
 * O(d n log n)); it touches no GPU.  Returns QMC_EINVAL for a composite or
 * out-of-range n. */
#ifndef __CUDACC_RTC__  /* function declarations are host-only */
int qmc_make_lattice(int32_t d, uint64_t n, const double* gamma, uint64_t* g_out);
#endif

/* The shifted rank-1 lattice rule, Eq. (2) and (3), on the GPU.
 *   d, n, m     dimension (1..QMC_DMAX), points (2 <= n < 2^31), shifts (2..1024)
 *   g           [d] generating vector, 1 <= g_i < n (host)
 *   shifts      [m * d] row-major shift table Delta_k in [0, 1) (host)
 *   t           transform
 *   f           integrand; f->d must equal d
 *   out         result (host or device)
 *   per_shift   optional [m * 2] array receiving Q^(k) (re, im), host or device
 *   stream      cudaStream_t
 * Returns QMC_EINVAL for bad arguments (m < 2, g_i outside [1, n), ...),
 * QMC_ECUDA if no GPU is usable, QMC_ENONFINITE / QMC_EDEFORM as warnings
 * (the estimate is still written) when `out` is host memory; with a device
 * `out` those two are reported in out->status only. */
#ifndef __CUDACC_RTC__  /* function declarations are host-only */
int qmc_integrate(int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts,
                  qmc_transform t, const qmc_integrand* f, qmc_result* out, double* per_shift,
                  void* stream);
#endif

/* A planned rule: the same arguments as qmc_integrate, validated and packed
 * once into launch descriptors and a device workspace owned by the plan, so
 * that qmc_plan_execute only launches kernels (no host staging, no
 * allocation). */
typedef struct qmc_plan_s* qmc_plan;
#ifndef __CUDACC_RTC__  /* function declarations are host-only */
int qmc_plan_create(int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts,
                    qmc_transform t, const qmc_integrand* f, qmc_plan* plan_out);
#endif
/* out / per_shift as for qmc_integrate.  Device memory keeps execute fully
 * asynchronous. */
#ifndef __CUDACC_RTC__  /* function declarations are host-only */
int qmc_plan_execute(qmc_plan plan, qmc_result* out, double* per_shift, void* stream);
int qmc_plan_destroy(qmc_plan plan);
#endif
/* Number of kernel launches one qmc_plan_execute issues. */
#ifndef __CUDACC_RTC__  /* function declarations are host-only */
int qmc_plan_launches(qmc_plan plan, int32_t* launches_out);
#endif
/* Autotuner: times the plan on `stream` with each specialised shift-chunk
 * size (shifts evaluated per point by one launch: 8, 16 or 32 for FP32EVAL
 * sector integrands, with register-pressure variants of the run-time
 * specialised kernel; other plans have one choice) and keeps the fastest.
 * QMC_TUNE_VERBOSE=1 in the environment prints each candidate's time to
 * stderr.  QMC_JIT_IMM=1 compiles the specialised kernel of a plan of one
 * launch chunk with its shift table as immediate operands of the coordinate
 * adds (one compilation per shift table; bit-identical results; measured
 * 5% slower on the benchmark's workload, so not a tuning candidate).
 * Reports the choice in *shifts_per_launch_out (may be NULL).  Synchronises
 * the device. */
#ifndef __CUDACC_RTC__  /* function declarations are host-only */
int qmc_plan_tune(qmc_plan plan, void* stream, int32_t* shifts_per_launch_out);
#endif
#ifndef __CUDACC_RTC__  /* function declarations are host-only */
/* One-line description of the plan's launches (kernel family, dimension,
 * shifts per launch, whether the kernel was specialised at run time for this
 * integrand, grid and tile size), NUL-terminated into buf[len]. */
int qmc_plan_describe(qmc_plan plan, char* buf, int32_t len);
#endif
/* Timing hook: when set (non-NULL cudaEvent_t handles passed as void*), every
 * later qmc_plan_execute records `before_rule` on its stream just before the
 * rule kernels and `after_rule` just after them (before the final pass), so a
 * caller can time the lattice kernels alone.  NULL, NULL clears the hook. */
#ifndef __CUDACC_RTC__  /* function declarations are host-only */
int qmc_plan_record_events(qmc_plan plan, void* before_rule, void* after_rule);
#endif

/* One problem of a batch: the arguments of qmc_integrate. */
typedef struct {
  int32_t d;
  int32_t m;
  uint64_t n;
  const uint64_t* g;
  const double* shifts;
  qmc_transform t;
  const qmc_integrand* f;
} qmc_problem;

/* Many independent rules (e.g. the sectors of one integral: uneven d, n,
 * integrand) evaluated together.  Every problem keeps the kernel it would get
 * from qmc_integrate, with at most ceil(n m / 2^16) CTAs (at most 4 per SM);
 * the problems' launches go round-robin to internal streams forked from
 * `stream` (the GPU runs the sectors side by side), followed by one
 * final-pass launch for all problems.  The workspace comes from the
 * stream-ordered allocator (cudaMallocAsync / cudaFreeAsync on `stream`).
 *   count      number of problems (1..65536)
 *   problems   [count] descriptors (host); each as for qmc_integrate
 *   out        [count] results (host or device); out[i].status per problem
 *   per_shift  optional; problem i writes 2*m_i doubles at offset 2*sum_{p<i} m_p
 * Synchronises `stream`.  Returns the first non-OK per-problem status when
 * `out` is host memory. */
#ifndef __CUDACC_RTC__  /* function declarations are host-only */
int qmc_integrate_batch(int32_t count, const qmc_problem* problems, qmc_result* out,
                        double* per_shift, void* stream);
#endif

/* Automatic choice of n for a batch (the sectors of one integral), each pass
 * one batched launch.  Problem i is first evaluated on its own lattice
 * (problems[i].n, .g), then on the ladder's lattices with n above its own, in
 * order; a ladder lattice serves every problem through its first d
 * components (a component-by-component vector of ladder_dim components
 * restricted to d is the d-dimensional one).  Each pass evaluates, as
 * qmc_integrate_batch would at their current lattices (bit for bit), only the
 * problems that move up; the others keep their last result.  Kernels,
 * shifts and coefficients are prepared once, so a pass costs its launches,
 * one final pass and one copy of the results.
 *   criterion QMC_WALK_SUM: stop when the sum's error estimate,
 *       sqrt(sum_i err_i^2), is <= rel_tol |sum_i Qbar_i|; else move up every
 *       problem whose err_i is above its share rel_tol |sum_i Qbar_i| / sqrt(count)
 *     QMC_WALK_EACH: stop when every problem meets err_i <= rel_tol |Qbar_i|;
 *       else move up every problem that does not
 *   (modulus of (re, im) for complex integrands).  Stops too when no problem
 *   that should move up has a further lattice.
 *   QMC_WALK_PERSISTENT (or-ed into criterion): each pass is one launch of a
 *   persistent kernel over work items of 2^15 points from all the problems
 *   it refines.  The kernel is specialised at run time per (problem, chunk of
 *   16 shifts) with the lattice as launch data, so one module serves every
 *   pass (built on first use, then cached).  Problems as for
 *   qmc_batch_plan_create_persistent (else QMC_EUNSUPPORTED); a problem's
 *   results equal that plan's at the same lattice, bit for bit.
 *   QMC_WALK_JUMP (or-ed into criterion): a problem that moves up goes to the
 *   first ladder lattice n' with (n'/n)^6 >= err_i / t_i, t_i its target
 *   (the share above, or rel_tol |Qbar_i|): as far as an error falling like
 *   n^-6 would need, instead of one lattice.  Errors that fall no faster
 *   than that (the rates the paper reports lie between n^-1 and n^-4) then
 *   never take a problem past the lattice it needs, and the lattices in
 *   between are skipped; estimates that fall faster can overshoot.  With
 *   t_i = 0 the problem moves one lattice.
 *   levels          ladder lattices (0..64), increasing n in [2, 2^31)
 *   ladder_n        [levels];  ladder_g  [levels * ladder_dim], g in [1, n)
 *   ladder_dim      components per ladder vector, >= every problem's d (when levels > 0)
 *   out             [count] results at the final lattices (host)
 *   level_out       optional [count]: ladder index of problem i's final
 *                   lattice, -1 for its own
 *   passes_out      optional: passes run
 * Synchronises `stream`.  Returns QMC_OK when the tolerance was met, else
 * QMC_ETIMEOUT with the last results (QMC_WALK_EACH: out[i].status =
 * QMC_ETIMEOUT for the problems that miss it); per-problem non-finite or
 * deformation warnings stay in out[i].status. */
#define QMC_WALK_SUM 0
#define QMC_WALK_EACH 1
#define QMC_WALK_PERSISTENT 0x10
#define QMC_WALK_JUMP 0x20
#ifndef __CUDACC_RTC__  /* function declarations are host-only */
int qmc_integrate_batch_to_tolerance(int32_t count, const qmc_problem* problems, int32_t levels,
                                     const uint64_t* ladder_n, const uint64_t* ladder_g, int32_t ladder_dim,
                                     double rel_tol, int32_t criterion, qmc_result* out, int32_t* level_out,
                                     int32_t* passes_out, void* stream);
#endif

/* Automatic choice of n for a batch on embedded base-2 lattices (Eq. 2 and
 * Eq. 3 as for qmc_integrate_extensible, the walk's passes and criterion as
 * for qmc_integrate_batch_to_tolerance).  Problem i starts with the rule of
 * problems[i].n = 2^k points whose vector is g mod 2^k (its first d
 * components; problems[i].g is not read).  A pass doubles the size of every
 * problem it refines and evaluates only the new points: the previous size's
 * lattice on shifts Delta_k + (g mod 2n) / (2n), averaged per shift with the
 * previous values, so each result is exactly the size-2n rule and no point is
 * evaluated twice.  All refined problems of a pass run as one batched launch.
 *   levels     most doublings per problem (0..30); no size exceeds 2^30
 *   g          [g_dim] odd components (qmc_make_lattice_embedded), host
 *   g_dim      >= every problem's d
 *   criterion  QMC_WALK_SUM or QMC_WALK_EACH, optionally | QMC_WALK_JUMP: a
 *              problem then takes the fewest k >= 1 doublings with
 *              64^k >= err_i / t_i in one pass, evaluating the whole rule of its new size when
 *              k > 1 (the points it had, at most a quarter of them, are
 *              evaluated again)
 *   level_out  optional [count]: doublings taken (final n = problems[i].n << level)
 * Problems as for qmc_integrate_batch, with m >= 2 and n a power of two in
 * [2, 2^30].  Synchronises `stream`.  Returns as
 * qmc_integrate_batch_to_tolerance; out[i].nonfinite and deform_violations
 * count every pass. */
#ifndef __CUDACC_RTC__  /* function declarations are host-only */
int qmc_integrate_batch_extensible(int32_t count, const qmc_problem* problems, int32_t levels, const uint64_t* g,
                                   int32_t g_dim, double rel_tol, int32_t criterion, qmc_result* out,
                                   int32_t* level_out, int32_t* passes_out, void* stream);
#endif

/* Planned batch: validates and packs once and builds the CUDA graph; every
 * execute replays it (one cudaGraphLaunch). */
typedef struct qmc_batch_plan_s* qmc_batch_plan;
#ifndef __CUDACC_RTC__  /* function declarations are host-only */
int qmc_batch_plan_create(int32_t count, const qmc_problem* problems, qmc_batch_plan* plan_out);
int qmc_batch_plan_execute(qmc_batch_plan plan, qmc_result* out, double* per_shift, void* stream);
int qmc_batch_plan_destroy(qmc_batch_plan plan);
#endif
/* The same batch as ONE persistent launch (the rule of Eq. (2) for every
 * problem, Eq. (3) per problem): CTAs take work items (problem, chunk of 8
 * shifts, chunk of `chunk_points` consecutive j) from a device counter, stage
 * the problem's rule into shared memory and sweep the chunk; item q of a
 * problem writes its fixed slots, so results do not depend on the order in
 * which CTAs take items.  Each problem must be an FP32EVAL SECTOR integrand
 * U^-2 F^-1 with deg U <= 1, deg F <= 2, d <= 8 and transform none, baker or
 * Korobov 3 (else QMC_EUNSUPPORTED).  The kernel is specialised at run time:
 * every (problem, chunk of up to 16 shifts) gets straight-line code with its
 * lattice, shifts and nonzero coefficients as constants (NVRTC, one program
 * per group of problems compiled on the host cores as relocatable code, then
 * linked into one module), and the persistent kernel dispatches each work
 * item to its problem's code.  When that is unavailable (no run-time
 * compilation, QMC_PERSIST_JIT=0 or QMC_JIT=0 in the environment, or more
 * than 60 KB of nonzero coefficient pairs for the module's constant bank),
 * one generic kernel stages each problem's dense coefficients in shared
 * memory instead (chunks of 8 shifts); qmc_batch_plan_describe reports which.
 * The plan replays one CUDA graph: counter reset, the persistent kernel, the
 * final pass.
 *   chunk_points  points per work item, a multiple of 256 in [256, 2^24];
 *                 0 = 65536 (qmc_batch_plan_tune sweeps 2^14..2^18)
 * Execute, launches, tune and destroy are those of qmc_batch_plan_create. */
#ifndef __CUDACC_RTC__  /* function declarations are host-only */
int qmc_batch_plan_create_persistent(int32_t count, const qmc_problem* problems, uint32_t chunk_points,
                                     qmc_batch_plan* plan_out);
#endif
/* One-line description of a batch plan, NUL-terminated into buf[len]: the
 * mode (graph or persistent); for a persistent plan whether its kernel was
 * specialised at run time, the descriptors (sector and shift chunk), work
 * items, CTAs, points per item and shift rows per descriptor. */
#ifndef __CUDACC_RTC__  /* function declarations are host-only */
int qmc_batch_plan_describe(qmc_batch_plan plan, char* buf, int32_t len);
#endif
/* Kernel launches in one replay (rule kernels + the final pass). */
#ifndef __CUDACC_RTC__  /* function declarations are host-only */
int qmc_batch_plan_launches(qmc_batch_plan plan, int32_t* launches_out);
#endif
/* Autotuner: times the graph on `stream` for evaluations-per-CTA budgets
 * 2^18..2^24 (the per-problem grid is ceil(n m / budget) CTAs), or, for a
 * persistent plan, for work items of 2^14..2^18 points (a specialised kernel
 * also built for two resident CTAs per SM, every function held to 128
 * registers), rebuilds the plan with the fastest and reports the work size in
 * *work_per_cta_out (may be NULL).
 * `problems` must describe the same batch the plan was created from.
 * Synchronises `stream`. */
#ifndef __CUDACC_RTC__  /* function declarations are host-only */
int qmc_batch_plan_tune(qmc_batch_plan plan, const qmc_problem* problems, void* stream,
                        uint64_t* work_per_cta_out);
#endif

/* Learned control variate (a separable rank-R cosine surrogate):
 *   g(z) = sum_{r<R} prod_{i<d} sum_{k<K} a[(r*d + i)*K + k] cos(F pi k z_i),
 *   int_[0,1]^d g = sum_r prod_i a[(r*d + i)*K]
 * fitted to the integrand f, so that Q^(k)[f - g] + int g, the rule of Eq. (2)
 * applied to f - g after the periodizing transform, is an unbiased estimate
 * with the same Eq. (3) error estimate.  This build: R = 16, K = 32, d <= 8.
 *   freq_step  F: 1 -> cos(pi k x); 2 -> cos(2 pi k x) (1-periodic basis)
 *   steps, lr  full-batch Adam (beta 0.9, 0.999), rate lr * (1 + cos(pi s/steps)) / 2
 *   band       0: every degree k < K is fitted; 1 <= band <= K: the degrees
 *              k >= band are held at zero (a band-limited surrogate, whose
 *              high derivatives, and so its content at the dual lattice's
 *              frequencies after the periodizing transform, stay small)
 *   seed       SplitMix64 seed of the initial parameters */
typedef struct {
  int32_t R;
  int32_t K;
  int32_t freq_step;
  int32_t steps;
  float lr;
  int32_t band;
  uint64_t seed;
} qmc_cv_config;

/* Fit the surrogate on the GPU to f at the n_pilot points of one shifted
 * lattice (g_pilot, shift_pilot [d]) on the untransformed cube (f evaluated in
 * FP64 by the rule's own kernel; t is not used here), mean squared error;
 * the fit's contractions run on tensor cores (BF16 operands, FP32
 * accumulation).
 *   a_out     [R*d*K] host, the parameters rounded to bfloat16 (stored as float)
 *   loss_out  optional [2] host: loss before the first and after the last step
 * Synchronises `stream`. */
#ifndef __CUDACC_RTC__  /* function declarations are host-only */
int qmc_cv_train(int32_t d, uint64_t n_pilot, const uint64_t* g_pilot, const double* shift_pilot,
                 qmc_transform t, const qmc_integrand* f, const qmc_cv_config* cfg, float* a_out,
                 double* loss_out, void* stream);
#endif

/* The rule with the control variate: one pass evaluates f and g at every
 * transformed point z(x) and sums both times the transform weight.
 * out->mean[0], var[0], err[0] are the control-variate estimate
 * Q[f - g] + int g; out->mean[1], var[1], err[1] the plain rule's Q[f] from
 * the same points (the fallback: keep whichever error is smaller).
 * per_shift (optional, [m*2]) gets the two per-shift values.  Supports
 * FP32EVAL sector integrands U^-2 F^-1 with deg U <= 1, deg F <= 2, d <= 8,
 * transform none, baker or Korobov 3.  f is evaluated as by the FP32 sector
 * kernels; g's per-dimension contraction runs on tensor cores (TF32 products
 * of the parameters with a head/remainder split of each basis value, degree 0
 * added in FP32), which keeps g to FP32 accuracy.  Engine: tcgen05.mma with
 * the basis written to tensor memory (one 128-point tile per MMA, M = 128,
 * N = 16), or warp-level mma.sync when QMC_CV_ENGINE=mma is set in the
 * environment.  The tcgen05 kernel's waits on its MMAs are bounded (about
 * 2 s); one that runs out makes the call return QMC_ETIMEOUT (out->status
 * too), and the context stays usable. */
#ifndef __CUDACC_RTC__  /* function declarations are host-only */
int qmc_integrate_cv(int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts,
                     qmc_transform t, const qmc_integrand* f, const qmc_cv_config* cfg, const float* a,
                     qmc_result* out, double* per_shift, void* stream);
#endif

/* Automatic choice of n with the control variate as a candidate (the ladder
 * of qmc_integrate_to_tolerance; the estimator of qmc_integrate_cv).  The
 * first min(3, levels) lattices are the pilot: on each, a control-variate
 * pass gives Q[f - g] + int g with its Eq. (3) error, and a plain pass
 * (qmc_integrate) the plain rule's.  Each estimator's convergence rate p
 * (relative error ~ n^-p) is the least-squares slope of log error against
 * log n over the pilot lattices (1 with a single lattice, clamped to
 * [1/4, 8]), and its time to reach rel_tol is predicted as its pass time on
 * the last pilot lattice times (error / rel_tol)^(1/p), the growth of n it
 * needs.  Both passes run once before they are timed, so first-use work (run-
 * time compilation) does not enter the comparison.  The estimator with the
 * smaller predicted time is kept for the rest of the ladder; the plain walk is
 * then exactly qmc_integrate_to_tolerance's.  A pilot lattice whose plain (or
 * else control-variate) estimate already meets rel_tol ends the walk there.
 * Stops at the first level whose kept estimate meets err / |Qbar| <= rel_tol.
 *   levels, n, g  as for qmc_integrate_to_tolerance
 *   cfg, a        the fitted surrogate (qmc_cv_train)
 *   out           host: the kept estimate in part [0] (part [1] zero for the
 *                 control variate; the plain result as is)
 *   level_out     the level that produced *out (may be NULL)
 *   mode_out      1 if the control variate was kept, 0 if the plain rule (may be NULL)
 *   judge_out     optional [8] host: on the last pilot lattice the relative
 *                 errors (control variate, plain) and pass times in seconds,
 *                 then the rates p (control variate, plain) and the predicted
 *                 times to rel_tol (control variate, plain)
 * Integrands as for qmc_integrate_cv.  Synchronises `stream`.  Returns QMC_OK
 * when the tolerance was met, else QMC_ETIMEOUT with the last level's
 * estimate. */
#ifndef __CUDACC_RTC__  /* function declarations are host-only */
int qmc_integrate_cv_to_tolerance(int32_t d, int32_t levels, const uint64_t* n, const uint64_t* g, int32_t m,
                                  const double* shifts, qmc_transform t, const qmc_integrand* f,
                                  const qmc_cv_config* cfg, const float* a, double rel_tol, qmc_result* out,
                                  int32_t* level_out, int32_t* mode_out, double* judge_out, void* stream);
#endif

/* The training kernels' loss and gradient at given parameters on given
 * points (x [P*d] in [0,1), targets h [P], host), for checking them against
 * an independent computation.  grad_out [R*d*K] host. */
#ifndef __CUDACC_RTC__  /* function declarations are host-only */
int qmc_cv_loss_grad(int32_t d, const qmc_cv_config* cfg, int32_t P, const double* x, const double* h,
                     const float* a, double* loss_out, float* grad_out, void* stream);
#endif

/* The rule of qmc_integrate without any device allocation, for callers that
 * cannot call cudaMalloc (code running where the CUDA allocator is locked,
 * exhausted or owned by a host framework, or inside host callbacks).  The
 * paper has no counterpart; this is an interface variant of qmc_integrate.
 * Scratch (per-CTA result slots, counters, result staging) comes from one
 * file-scope device array of 4 MiB per device, resident until the process
 * exits.  Its address is looked up once per device, with that device
 * current, by the first call on that device; make that first call before any
 * stream capture.  Under CUDA's lazy module loading (the default) that first
 * call is also what loads the library's module on the device and so
 * reserves the 4 MiB there: a caller that expects its allocator to be
 * exhausted or locked later should make one small call on each device while
 * device memory is still available.  Every call shares the array and leaves its contents
 * behind (the counters are cleared at the start of each call), so calls
 * whose GPU work overlaps (different streams or host threads) race on it:
 * order them.  Supports SECTOR integrands U^-2 F^-1 with deg U <= 1,
 * deg F <= 2, d <= 8 (FP64 or FP32EVAL; Korobov weight 3, baker or none).
 * Returns QMC_EINVAL when m x (CTAs of one resident wave) slots exceed the
 * fixed array, QMC_EUNSUPPORTED for other integrands.  Arguments, outputs and
 * synchronisation as for qmc_integrate. */
#ifndef __CUDACC_RTC__  /* function declarations are host-only */
int qmc_integrate_noalloc(int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts,
                          qmc_transform t, const qmc_integrand* f, qmc_result* out, double* per_shift,
                          void* stream);
#endif

/* Single terms of Eq. (2), evaluated by the same device code the rule uses:
 * for each sample s, the weighted value f(z(x)) prod_i w(x_i) at point
 * j[s] (0-based, the paper's j-1) and shift k[s].
 *   values  [count * 2] (re, im), host
 *   idx     optional [count * d] lattice indices (j g_i) mod n, host
 *   coord   optional [count * d] the coordinate x the kernel used, as double, host
 * Synchronises `stream`. */
#ifndef __CUDACC_RTC__  /* function declarations are host-only */
int qmc_sample_points(int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts,
                      qmc_transform t, const qmc_integrand* f, int32_t count, const uint64_t* j,
                      const int32_t* k, double* values, uint64_t* idx, double* coord, void* stream);
#endif

#ifndef __CUDACC_RTC__  /* function declarations are host-only */
/* Automatic choice of n: applies the rule (Eq. 2, 3) on the lattices
 * (n[l], g[l * d ...]) for l = 0, 1, ... in turn and stops at the first whose
 * error estimate satisfies err / |Qbar| <= rel_tol (real part, or modulus for
 * complex integrands), or after the last.
 *   levels       number of lattices (1..64), increasing n
 *   n            [levels] lattice sizes;  g  [levels * d] generating vectors (host)
 *   level_out    index of the lattice that produced *out
 * The shifts, transform and integrand are those of qmc_integrate; `out`
 * must be host memory.  Returns QMC_OK if the tolerance was met, else the
 * last level's estimate with status QMC_ETIMEOUT in out->status and as the
 * return value. */
int qmc_integrate_to_tolerance(int32_t d, int32_t levels, const uint64_t* n, const uint64_t* g, int32_t m,
                               const double* shifts, qmc_transform t, const qmc_integrand* f, double rel_tol,
                               qmc_result* out, int32_t* level_out, void* stream);
#endif

#ifndef __CUDACC_RTC__  /* function declarations are host-only */
/* Embedded rank-1 lattices in base 2 (automatic n without discarding work).
 * One generating vector g serves every size 2^k, log2_nmin <= k <= log2_nmax:
 * the size-2^k lattice is {j g / 2^k}, the points of size 2n include those of
 * size n, and the others form the size-n lattice shifted by g / (2n).
 * qmc_make_lattice_embedded builds g component by component (g_1 = 1, odd
 * components) minimising max_k 4^k e^2_{2^k}(g), with e^2 the worst-case
 * error of qmc_make_lattice at each size.  When `candidates` covers all odd
 * z < 2^(log2_nmax - 1), all of them are searched at once (cyclic correlations
 * over the powers of 5 by FFT, O(N log N) per component, the best few then
 * recomputed exactly); otherwise `candidates` odd z drawn by SplitMix64 from
 * `seed` are evaluated directly.  Ties go to the smallest z.  Host only; sizes
 * up to 2^30.  g_out: [d] host. */
int qmc_make_lattice_embedded(int32_t d, int32_t log2_nmin, int32_t log2_nmax, const double* gamma,
                              int32_t candidates, uint64_t seed, uint64_t* g_out);
/* Doubling n until Eq. (3)'s relative error meets rel_tol: level 0 applies the
 * rule with n = 2^log2_n0 points; level l >= 1 evaluates only the new points
 * of n = 2^(log2_n0 + l), as the rule of the previous size on shifts
 * Delta + g / n, and averages it with the previous per-shift values, so the
 * estimate at every level is exactly the size-2^(log2_n0 + l) rule.
 *   levels     1..31 - log2_n0 sizes;  g [d] odd components, for the largest size
 *   per_shift  optional [m][2] host: the per-shift values of the returned level
 *   level_out  the level that produced *out
 * Shifts, transform and integrand as for qmc_integrate; `out` is host memory.
 * Returns QMC_OK when the tolerance was met (or the level's NaN/Inf warning),
 * else the last level's estimate with status QMC_ETIMEOUT. */
int qmc_integrate_extensible(int32_t d, int32_t log2_n0, int32_t levels, const uint64_t* g, int32_t m,
                             const double* shifts, qmc_transform t, const qmc_integrand* f, double rel_tol,
                             qmc_result* out, double* per_shift, int32_t* level_out, void* stream);
#endif

#ifndef __CUDACC_RTC__  /* function declarations are host-only */
/* Eq. (2)/(3) from per-shift values alone: Qbar and sigma^2 (two-pass,
 * compensated) over m values Q^(k) given as per_shift [m][2] (re, im), host
 * memory; host only, no GPU.  Combines independent shift sets (from several
 * GPUs, or earlier and later calls that append shifts) into one estimate.
 * Returns QMC_EINVAL for m < 2. */
int qmc_combine_shifts(int32_t m, const double* per_shift, qmc_result* out);
#endif

#ifndef __CUDACC_RTC__  /* function declarations are host-only */
/* Measured arithmetic peaks of the current GPU, out[4]: out[0] FP32 FMA
 * TFLOP/s, out[1] FP64 FMA TFLOP/s (independent dependency chains on a full
 * grid), out[2] warp-level TF32 mma.sync m16n8k8 TFLOP/s and out[3] warp-level
 * BF16 mma.sync m16n8k16 TFLOP/s (the instructions of the control variate's
 * estimator and fit; 8 independent accumulators per warp); each the best of
 * 5, CUDA events on `stream`.
 * A measurement utility beside the rule; synchronises `stream`. */
int qmc_measure_peaks(void* stream, double* out);
#endif

/* Epsilon expansion of the sector integrand (Eq. 7 with regulated powers,
 * Sec. 2): for U^(aU + bU eps) F^(aF + bF eps) = sum_k eps^k f_k,
 *   f_k = U^aU F^aF L^k / k!,  L = bU log U + bF log F,
 * one pass over the lattice estimates f_0 .. f_{orders-1} together: the
 * point, transform, U and F are computed once per (point, shift) and shared
 * by all orders.  f_0 is the SECTOR integrand itself (eps = 0).
 *   orders  1..QMC_EPS_MAX coefficient integrands
 *   bU, bF  finite slopes of the powers in eps (U^(-2+eps) F^(-1-eps): 1, -1)
 * Values where U <= 0 or F <= 0 make L NaN; each order counts and leaves out
 * its own non-finite values (out[o].nonfinite, status QMC_ENONFINITE). */
#define QMC_EPS_MAX 6
typedef struct {
  int32_t orders;
  int32_t reserved;
  double bU;
  double bF;
} qmc_eps;

#ifndef __CUDACC_RTC__  /* function declarations are host-only */
/* Eq. (2)/(3) for every order.  Arguments as qmc_integrate, f->kind must be
 * QMC_F_SECTOR (else QMC_EINVAL), and
 *   out        [orders] results, order o in out[o] (host or device)
 *   per_shift  optional [orders][m][2] Q^(k) per order
 * Returns the first non-OK status of the orders when `out` is host memory. */
int qmc_integrate_eps(int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts,
                      qmc_transform t, const qmc_integrand* f, const qmc_eps* eps, qmc_result* out,
                      double* per_shift, void* stream);
/* A plan of the same (see qmc_plan_create); qmc_plan_execute on it writes
 * out[orders] and per_shift [orders][m][2]. */
int qmc_eps_plan_create(int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts,
                        qmc_transform t, const qmc_integrand* f, const qmc_eps* eps, qmc_plan* plan_out);
/* Single terms: values [count][orders] (host), order o of the weighted value
 * at point j[s], shift k[s], by the device code of qmc_integrate_eps.
 * Synchronises `stream`. */
int qmc_sample_points_eps(int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts,
                          qmc_transform t, const qmc_integrand* f, const qmc_eps* eps, int32_t count,
                          const uint64_t* j, const int32_t* k, double* values, void* stream);
#endif

/* Several integrands on one lattice.  The sectors of one dimension that share
 * (n, g, shifts, transform) are evaluated in one sweep (Eq. 2 for each): the
 * lattice index, fixed-point base and transformed coordinates of every
 * (point, shift) are computed once and shared by all of them.  The sum of
 * the integrands is reported too: its per-shift values are the sums of the
 * integrands' per-shift values, and Eq. (3) is applied to those.
 *   count      1..QMC_MULTI_MAX integrands fs[0..count-1], each QMC_F_SECTOR
 *              of dimension d (<= 8), precision QMC_FP32EVAL, U of degree <= 1,
 *              F of degree <= 2, powers aU = -2, aF = -1
 *   transform  baker, Korobov 3 or none
 *   out        [count + 1] results: out[s] for fs[s], out[count] for the sum
 *              (host or device)
 *   per_shift  optional [(count + 1)][m][2]
 * The fused kernel is specialised at run time for the integrands' monomials
 * (NVRTC); without run-time compilation the call returns QMC_EUNSUPPORTED.
 * Other requests return QMC_EINVAL (bad arguments) or QMC_EUNSUPPORTED. */
#define QMC_MULTI_MAX 256
#ifndef __CUDACC_RTC__  /* function declarations are host-only */
int qmc_integrate_multi(int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts,
                        qmc_transform t, int32_t count, const qmc_integrand* fs, qmc_result* out,
                        double* per_shift, void* stream);
/* A plan of the same; qmc_plan_execute on it writes out[count + 1] and
 * per_shift [(count + 1)][m][2]. */
int qmc_multi_plan_create(int32_t d, uint64_t n, int32_t m, const uint64_t* g, const double* shifts,
                          qmc_transform t, int32_t count, const qmc_integrand* fs, qmc_plan* plan_out);
#endif

/* Text of the last error raised on the calling thread ("" if none). */
#ifndef __CUDACC_RTC__  /* function declarations are host-only */
const char* qmc_last_error(void);
#endif

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
#ifndef __CUDACC_RTC__  /* function declarations are host-only */
int32_t qmc_version(void);
#endif

#ifdef __cplusplus
}
#endif

#endif /* QMC_H */

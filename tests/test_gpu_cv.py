"""GPU parity of the control-variate estimator Q[f - g] + int g (tensor-core
surrogate: cv_tc_kernel with warp-level MMA, cv_tc5_kernel with tcgen05 and
the basis in tensor memory) against the oracle, for every transform it takes.

Tolerances.  h = f(z) prod w is the FP32 sector path's value (per shift the
oracle's Q^(k)[h] within 2e-7 relative, as for the plain FP32 path).  The
surrogate g is evaluated with FP32 cosines, an FP32 Chebyshev recurrence,
and TF32 products on a head/remainder split of each basis value (about 22
bits kept) with FP32 accumulation: per point a relative error of a few 1e-7
at most, averaging out over the lattice.  The per-shift control-variate
value is therefore held to 2e-7 of (|Q^(k)[h]| + |int g|), its two parts'
scale, and the surrogate's own quadrature error int g - Q^(k)[g] (the
difference of the two per-shift results, which cancels h) to 5e-8 of
|int g|: a surrogate evaluated with a BF16 basis (8 bits) or with a dropped
remainder would miss it by orders of magnitude."""

import numpy as np
import pytest

from paper_1811_11722_gb300 import inputs as I

pytestmark = pytest.mark.gpu

R, K = 16, 32


@pytest.fixture(scope="module")
def Q():
    from paper_1811_11722_gb300 import build, qmc
    build.build_library()
    return qmc


@pytest.fixture(params=["mma", "tcgen05"])
def engine(request, monkeypatch):
    """The estimator's contraction: warp-level mma.sync (cv_tc_kernel) or
    tcgen05.mma with the basis in tensor memory (cv_tc5_kernel, the default)."""
    monkeypatch.setenv("QMC_CV_ENGINE", request.param)
    return request.param


def _cfg(Q, steps=300, freq=1, seed=7):
    cfg = Q.qmc_cv_config()
    cfg.R, cfg.K, cfg.freq_step, cfg.steps, cfg.lr, cfg.seed = R, K, freq, steps, 1e-2, seed
    return cfg


def _problem(d, n, m, transform, seed):
    """A degree-(1, 2) sector integrand U^-2 F^-1 in d dimensions."""
    rng = I.SplitMix64(seed)
    U = I.random_poly(rng, d, min(d, 4), 0)
    F = I.random_poly(rng, d, 0, min(3 * d, 12))
    shifts = I.make_shifts(rng, m, d)
    alpha = 3 if transform == "korobov" else 0
    return I.Problem(f"cv_d{d}", d, n, m, shifts, transform, alpha=alpha, kind="sector", U=U, F=F,
                     aU=-2, aF=-1, precision="fp32", gamma=I.product_weights(d))


def _params(oracle_lib, d, seed):
    """Surrogate parameters as bfloat16 values: constant terms near 1 (so g
    is of the integrand's order), the rest N(0, 0.03)."""
    rng = np.random.default_rng(seed)
    a = rng.normal(0.0, 0.03, size=(R, d, K))
    a[:, :, 0] = 0.55 + 0.1 * rng.random((R, d))
    return np.array([oracle_lib.bf16(v) for v in a.ravel()], dtype=np.float32)


def _transform(Q, p):
    return Q.transform(p.transform, p.alpha)


@pytest.mark.parametrize("d,transform,n,m", [
    (8, "none", 30011, 3),       # ragged tail, one partial shift chunk
    (8, "korobov", 50021, 10),   # two launches, the second partial
    (5, "baker", 65521, 4),
    (3, "korobov", 20011, 9),
    (1, "baker", 10007, 2),
])
def test_cv_estimator_matches_oracle(Q, oracle_lib, nthreads, engine, d, transform, n, m):
    p = _problem(d, n, m, transform, seed=100 + d)
    g = I.random_generating_vector(I.SplitMix64(200 + d), d, n)
    a = _params(oracle_lib, d, seed=300 + d)
    f = Q.integrand_from_problem(p, "fp32")
    res, ps = Q.qmc_integrate_cv(d, n, m, g, p.shifts, _transform(Q, p), f, _cfg(Q), a)
    assert res.as_dict()["status"] == 0
    gint = oracle_lib.cv_integral(d, R, K, a)
    ref_plain = oracle_lib.integrate(p, g, nthreads=nthreads)["q"][:, 0]
    p.cv = {"R": R, "K": K, "F": 1, "a": a}
    ref_cv = oracle_lib.integrate(p, g, nthreads=nthreads)["q"][:, 0] + gint
    scale = np.abs(ref_plain) + abs(gint)
    dev_plain = np.max(np.abs(ps[:, 1] - ref_plain) / np.abs(ref_plain))
    dev_cv = np.max(np.abs(ps[:, 0] - ref_cv) / scale)
    # the surrogate alone: int g - Q^(k)[g] from both sides
    quad_gpu = ps[:, 0] - ps[:, 1]
    quad_ref = ref_cv - ref_plain
    dev_quad = np.max(np.abs(quad_gpu - quad_ref)) / abs(gint)
    print(f"{engine} d={d} {transform} n={n}: plain {dev_plain:.2e}, cv {dev_cv:.2e}, surrogate quadrature {dev_quad:.2e} "
          f"(int g - Q[g] ~ {np.max(np.abs(quad_ref)) / abs(gint):.1e} of int g)")
    assert dev_plain <= 2e-7
    assert dev_cv <= 2e-7
    assert dev_quad <= 5e-8


def test_cv_estimator_freq2_and_zero_surrogate(Q, oracle_lib, nthreads, engine):
    """The cos(2 pi k z) basis against the oracle; and a surrogate that is
    identically zero gives the plain rule's values exactly (same h, nothing
    subtracted)."""
    d, n, m = 4, 30011, 3
    p = _problem(d, n, m, "baker", seed=77)
    g = I.random_generating_vector(I.SplitMix64(78), d, n)
    a = _params(oracle_lib, d, seed=79)
    f = Q.integrand_from_problem(p, "fp32")
    _, ps = Q.qmc_integrate_cv(d, n, m, g, p.shifts, _transform(Q, p), f, _cfg(Q, freq=2), a)
    gint = oracle_lib.cv_integral(d, R, K, a)
    ref_plain = oracle_lib.integrate(p, g, nthreads=nthreads)["q"][:, 0]
    p.cv = {"R": R, "K": K, "F": 2, "a": a}
    ref_cv = oracle_lib.integrate(p, g, nthreads=nthreads)["q"][:, 0] + gint
    assert np.max(np.abs(ps[:, 0] - ref_cv) / (np.abs(ref_plain) + abs(gint))) <= 2e-7
    assert np.max(np.abs((ps[:, 0] - ps[:, 1]) - (ref_cv - ref_plain))) <= 5e-8 * abs(gint)
    z = np.zeros_like(a)
    _, ps0 = Q.qmc_integrate_cv(d, n, m, g, p.shifts, _transform(Q, p), f, _cfg(Q, freq=2), z)
    assert np.array_equal(ps0[:, 0], ps0[:, 1])
    assert np.max(np.abs(ps0[:, 1] - ref_plain) / np.abs(ref_plain)) <= 2e-7


def test_cv_gain_by_transform(Q):
    """What the trained surrogate gains over the rule without it, from the
    same points (configuration-5 integrand, d = 8, n = 1048573, m = 16; one
    fit, 2000 Adam steps).  Without a periodising transform the rule's error
    comes from the integrand's non-periodicity, which the surrogate (fitted
    on the cube) takes out: the control variate's Eq. (3) error is several
    times smaller.  With the Korobov transform the rule already converges
    fast and the surrogate's own dual-lattice content dominates: it loses.
    The ratios are printed for the record; the gain without a transform is
    asserted."""
    p = I.config5(n=1048573, m=16)
    g = Q.qmc_make_lattice(8, p.n, p.gamma)
    gp = Q.qmc_make_lattice(8, 65537, p.gamma)
    f = Q.integrand_from_problem(p, "fp32")
    cfg = _cfg(Q, steps=2000)
    a, losses = Q.qmc_cv_train(8, 65537, gp, I.make_shifts(I.SplitMix64(54), 1, 8)[0], Q.transform("none"), f, cfg)
    gains = {}
    for name, t in (("none", Q.transform("none")), ("baker", Q.transform("baker")),
                    ("korobov3", Q.transform("korobov", 3))):
        r = Q.qmc_integrate_cv(p.d, p.n, p.m, g, p.shifts, t, f, cfg, a)[0].as_dict()
        assert abs(r["mean"][0] - r["mean"][1]) <= 6 * (r["err"][0] + r["err"][1])
        gains[name] = r["err"][1] / r["err"][0]
        print(f"{name}: err cv {r['err'][0]:.3e} plain {r['err'][1]:.3e} gain {gains[name]:.2f}")
    assert gains["none"] >= 2.0


@pytest.mark.slow
def test_cv_estimator_full_size(Q, oracle_lib, nthreads, engine):
    """The estimator at the size the benchmark times it (configuration-5
    integrand, d = 8, Korobov 3, n = 16777213; two shifts, one launch): both
    per-shift sums against the oracle over all 16.7M points, and the
    surrogate's own quadrature int g - Q^(k)[g] to 5e-8 of int g, as for the
    small cases."""
    p = I.with_shifts(I.config5(n=16777213, m=2), 2, 61)
    g = Q.qmc_make_lattice(8, p.n, p.gamma)
    a = _params(oracle_lib, 8, seed=62)
    f = Q.integrand_from_problem(p, "fp32")
    _, ps = Q.qmc_integrate_cv(8, p.n, p.m, g, p.shifts, Q.transform("korobov", 3), f, _cfg(Q), a)
    gint = oracle_lib.cv_integral(8, R, K, a)
    ref_plain = oracle_lib.integrate(p, g, nthreads=nthreads)["q"][:, 0]
    p.cv = {"R": R, "K": K, "F": 1, "a": a}
    ref_cv = oracle_lib.integrate(p, g, nthreads=nthreads)["q"][:, 0] + gint
    dev_plain = np.max(np.abs(ps[:, 1] - ref_plain) / np.abs(ref_plain))
    dev_cv = np.max(np.abs(ps[:, 0] - ref_cv) / (np.abs(ref_plain) + abs(gint)))
    dev_quad = np.max(np.abs((ps[:, 0] - ps[:, 1]) - (ref_cv - ref_plain))) / abs(gint)
    print(f"{engine} full size: plain {dev_plain:.2e}, cv {dev_cv:.2e}, surrogate quadrature {dev_quad:.2e}")
    assert dev_plain <= 2e-7 and dev_cv <= 2e-7 and dev_quad <= 5e-8


def test_band_limited_fit_holds_high_degrees_at_zero(Q):
    """cfg.band = 8: the fitted parameters of degrees k >= 8 are exactly zero
    (bfloat16 zeros), the others are trained, and int g stays the product of
    the constant terms (the estimator is unchanged)."""
    d = 3
    p = _problem(d, 4099, 2, "korobov", seed=41)
    f = Q.integrand_from_problem(p, "fp32")
    gp = Q.qmc_make_lattice(d, 4099, I.product_weights(d))
    cfg = _cfg(Q, steps=200)
    cfg.band = 8
    a, losses = Q.qmc_cv_train(d, 4099, gp, I.make_shifts(I.SplitMix64(3), 1, d)[0], Q.transform("none"), f, cfg)
    a = a.reshape(R, d, K)
    assert np.all(a[:, :, 8:] == 0.0)
    assert np.any(a[:, :, 1:8] != 0.0)
    assert losses[1] < losses[0]
    cfg.band = K + 1
    with pytest.raises(Q.QmcError):
        Q.qmc_cv_train(d, 4099, gp, I.make_shifts(I.SplitMix64(3), 1, d)[0], Q.transform("none"), f, cfg)


def _ladder(Q, d, ns, gamma):
    return np.concatenate([Q.qmc_make_lattice(d, n, gamma) for n in ns])


def test_cv_walk_falls_back_to_the_plain_rule(Q):
    """The control-variate walk judges the surrogate on the first three
    lattices by predicted time to the target.  On the configuration-5
    integrand under Korobov 3 the plain rule's error falls much faster with n
    than the control variate's, so the walk keeps the plain rule (mode 0),
    and it is exactly the plain walk: same stopping level, same estimate as
    qmc_integrate_to_tolerance on the same ladder."""
    p = I.config5(n=65521, m=16)
    d = p.d
    ns = [65521, 131071, 262139, 524287, 1048573, 2097143]
    gs = _ladder(Q, d, ns, p.gamma)
    f = Q.integrand_from_problem(p, "fp32")
    t = Q.transform("korobov", 3)
    gp = Q.qmc_make_lattice(d, I.N_PILOT, p.gamma)
    cfg = _cfg(Q, steps=400)
    a, _ = Q.qmc_cv_train(d, I.N_PILOT, gp, I.make_shifts(I.SplitMix64(54), 1, d)[0], Q.transform("none"), f, cfg)
    tol = 1e-7
    r, lvl, mode, judge, ok = Q.qmc_integrate_cv_to_tolerance(d, ns, gs, p.m, p.shifts, t, f, cfg, a, tol)
    assert mode == 0, judge
    assert judge["predicted_s_cv"] >= judge["predicted_s_plain"]
    assert judge["rate_plain"] > judge["rate_cv"]
    r2, lvl2, ok2 = Q.qmc_integrate_to_tolerance(d, ns, gs, p.m, p.shifts, t, f, tol)
    assert (lvl, ok) == (lvl2, ok2)
    assert r.mean[0] == r2.mean[0] and r.err[0] == r2.err[0]


def test_cv_walk_keeps_a_winning_surrogate(Q):
    """Where the surrogate wins the walk keeps it (mode 1): a d = 1 sector
    without a transform, which 32 cosines fit to about 1e-9, so the control
    variate's error is orders of magnitude below the plain rule's at the
    same rate (both decay as about 1/n here, the non-periodic integrand's
    rate), and its predicted time to the target is far smaller.  The kept
    estimate is the control variate's, Q[f - g] + int g, with its own Eq. (3)
    error."""
    d = 1
    U = I.Poly(np.array([0.7, 1.3]), np.array([[0], [1]], dtype=np.uint8))
    F = I.Poly(np.array([0.4, 1.9]), np.array([[0], [2]], dtype=np.uint8))
    rng = I.SplitMix64(61)
    p = I.Problem("d1cv", 1, 65521, 8, I.make_shifts(rng, 8, 1), "none", kind="sector", U=U, F=F, precision="fp32")
    f = Q.integrand_from_problem(p, "fp32")
    t = Q.transform("none")
    ns = [10007, 20011, 40009, 80021]
    gs = np.ones(len(ns), dtype=np.uint64)
    gp = np.array([1], dtype=np.uint64)
    cfg = _cfg(Q, steps=2000)
    a, losses = Q.qmc_cv_train(d, 65537, gp, np.array([0.25]), t, f, cfg)
    r, lvl, mode, judge, ok = Q.qmc_integrate_cv_to_tolerance(d, ns, gs, p.m, p.shifts, t, f, cfg, a, 1e-11)
    assert mode == 1, (judge, losses)
    if lvl >= 2:  # past the first lattices the judgement was made on predicted times
        assert judge["predicted_s_cv"] < judge["predicted_s_plain"], judge
    rc, _ = Q.qmc_integrate_cv(d, ns[lvl], p.m, gs[lvl:lvl + 1], p.shifts, t, f, cfg, a)
    assert r.mean[0] == rc.mean[0] and r.err[0] == rc.err[0]


def test_tcgen05_wait_runs_out_and_reports(Q, oracle_lib, monkeypatch):
    """The tcgen05 estimator's waits are bounded.  With no MMA issued
    (QMC_CV_TEST_STALL=1) every wait on the MMA's mbarrier runs out: the
    kernel's groups leave together, free their tensor memory and flag the
    launch, and the call returns QMC_ETIMEOUT.  The next call on the same
    context gives the same values as the call before."""
    monkeypatch.setenv("QMC_CV_ENGINE", "tcgen05")
    d, n, m = 2, 1009, 2
    p = _problem(d, n, m, "baker", seed=5)
    g = I.random_generating_vector(I.SplitMix64(6), d, n)
    a = _params(oracle_lib, d, seed=7)
    f = Q.integrand_from_problem(p, "fp32")
    args = (d, n, m, g, p.shifts, _transform(Q, p), f, _cfg(Q), a)
    before = Q.qmc_integrate_cv(*args)[1]
    monkeypatch.setenv("QMC_CV_TEST_STALL", "1")
    with pytest.raises(Q.QmcError) as ei:
        Q.qmc_integrate_cv(*args)
    assert ei.value.status == Q.QMC_ETIMEOUT
    monkeypatch.delenv("QMC_CV_TEST_STALL")
    after = Q.qmc_integrate_cv(*args)[1]
    assert np.array_equal(before, after)

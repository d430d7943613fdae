"""GPU parity of the shared-lattice sweep: several sector integrands of one
dimension on the same (n, g, shifts, transform), evaluated by one fused
kernel, against the oracle for each integrand and for their sum.

Tolerances are those of the FP32EVAL path (per-shift Q^(k) within 2e-7
relative of the oracle).  Against the single-integrand kernel the per-point
values are the same floating-point operations in the same order, so only
the grouping of the compensated run sums differs (1e-8 relative)."""
import numpy as np
import pytest

from paper_1811_11722_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    from paper_1811_11722_gb300 import build, qmc
    build.build_library()
    return qmc


def oracle_sum(oracle_lib, probs, g, nthreads=1):
    """Per-integrand oracle results and the sum's Eq. (2)/(3) from the summed
    per-shift sums."""
    refs = [oracle_lib.integrate(p, g, nthreads=nthreads) for p in probs]
    sums = np.sum([r["sums"] for r in refs], axis=0)
    q, mean, var = oracle_lib.estimate(sums, probs[0].n)
    return refs, {"q": q, "mean": mean, "err": np.sqrt(var)}


@pytest.mark.parametrize("transform,alpha", [("baker", 0), ("korobov", 3), ("none", 0)])
def test_multi_vs_oracle(Q, oracle_lib, nthreads, transform, alpha):
    """11 integrands (a full chunk of 8 and a ragged chunk of 3), d = 6,
    n = 100003 (many tiles, ragged tail), m = 9 (an odd last shift pair)."""
    probs = I.config3_shared(count=11, d=6, n=100003, m=9, transform=transform, alpha=alpha)
    g = I.random_generating_vector(I.SplitMix64(61), 6, probs[0].n)
    fs = [Q.integrand_from_problem(p, "fp32") for p in probs]
    res, ps = Q.qmc_integrate_multi(6, probs[0].n, 9, g, probs[0].shifts, Q.transform(transform, alpha), fs,
                                    want_per_shift=True)
    assert len(res) == 12
    refs, tot = oracle_sum(oracle_lib, probs, g, nthreads)
    for s in range(11):
        assert res[s].status == 0 and res[s].nonfinite == 0
        assert np.all(np.abs(ps[s, :, 0] - refs[s]["q"][:, 0]) <= 2e-7 * np.abs(refs[s]["q"][:, 0])), s
        assert abs(res[s].mean[0] - refs[s]["mean"][0]) <= 2e-7 * abs(refs[s]["mean"][0]), s
    assert np.all(np.abs(ps[11, :, 0] - tot["q"][:, 0]) <= 2e-7 * np.abs(tot["q"][:, 0]))
    assert abs(res[11].mean[0] - tot["mean"][0]) <= 2e-7 * abs(tot["mean"][0])
    # the sum's per-shift values are the integrands' per-shift values added
    assert np.allclose(ps[11, :, 0], ps[:11, :, 0].sum(axis=0), rtol=1e-13, atol=0)


def test_multi_matches_single_integrand_kernel(Q):
    """The fused sweep against one qmc_integrate per integrand (d = 8, two chunks)."""
    probs = I.config3_shared(count=16, d=8, n=1000003, m=16)
    g = I.random_generating_vector(I.SplitMix64(62), 8, probs[0].n)
    fs = [Q.integrand_from_problem(p, "fp32") for p in probs]
    t = Q.transform("baker")
    res, ps = Q.qmc_integrate_multi(8, probs[0].n, 16, g, probs[0].shifts, t, fs, want_per_shift=True)
    for s, f in enumerate(fs):
        one, ps1 = Q.qmc_integrate(8, probs[0].n, 16, g, probs[0].shifts, t, f, want_per_shift=True)
        assert np.all(np.abs(ps[s, :, 0] - ps1[:, 0]) <= 1e-8 * np.abs(ps1[:, 0])), s
        assert abs(res[s].err[0] - one.err[0]) <= 1e-3 * one.err[0] + 1e-9 * abs(one.mean[0]), s


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 7])
def test_multi_all_dims(Q, oracle_lib, d):
    probs = I.config3_shared(count=5, d=d, n=20011, m=4, transform="korobov", alpha=3)
    g = I.random_generating_vector(I.SplitMix64(63 + d), d, probs[0].n)
    fs = [Q.integrand_from_problem(p, "fp32") for p in probs]
    res, ps = Q.qmc_integrate_multi(d, probs[0].n, 4, g, probs[0].shifts, Q.transform("korobov", 3), fs,
                                    want_per_shift=True)
    refs, tot = oracle_sum(oracle_lib, probs, g)
    for s in range(5):
        assert np.all(np.abs(ps[s, :, 0] - refs[s]["q"][:, 0]) <= 4e-7 * np.abs(refs[s]["q"][:, 0])), (d, s)
    assert np.all(np.abs(ps[5, :, 0] - tot["q"][:, 0]) <= 4e-7 * np.abs(tot["q"][:, 0]))


def test_multi_nonfinite_counted_per_integrand(Q, oracle_lib):
    """One integrand's F has no constant term, so 1/F is infinite where z = 0;
    it counts those points, the others count none, the sum counts them all."""
    d, n, m = 2, 1009, 4
    rng = I.SplitMix64(64)
    sh = I.make_shifts(rng, m, d)
    sh[0] = 0.0
    good = [I.Problem(f"ok{s}", d, n, m, sh, "baker", kind="sector", U=I.random_poly(rng, d, 2, 0),
                      F=I.random_poly(rng, d, 0, 3)) for s in range(3)]
    bad = I.Problem("nf", d, n, m, sh, "baker", kind="sector",
                    U=I.Poly(np.array([1.0]), np.zeros((1, d), np.uint8)),
                    F=I.Poly(np.array([1.0, 1.0]), np.array([[2, 0], [0, 2]], np.uint8)))
    probs = good[:2] + [bad] + good[2:]
    g = np.array([1, 17], dtype=np.uint64)
    fs = [Q.integrand_from_problem(p, "fp32") for p in probs]
    res, ps = Q.qmc_integrate_multi(d, n, m, g, sh, Q.transform("baker"), fs, want_per_shift=True)
    refs = [oracle_lib.integrate(p, g) for p in probs]
    nf = int(refs[2]["nonfinite"].sum())
    assert nf > 0
    for s in range(4):
        assert res[s].nonfinite == int(refs[s]["nonfinite"].sum()), s
    assert res[2].status == Q.QMC_ENONFINITE and res[0].status == 0
    assert res[4].nonfinite == nf and res[4].status == Q.QMC_ENONFINITE
    # 1/F ~ 1/|z|^2 near the left-out point: FP32 coordinates (2^-24 absolute)
    # put ~2 dz/|z| relative error on such values, so the comparison is with the
    # single-integrand FP32 kernel, which does the same arithmetic
    one, ps1 = Q.qmc_integrate(d, n, m, g, sh, Q.transform("baker"), fs[2], want_per_shift=True)
    assert one.nonfinite == nf
    assert np.all(np.abs(ps[2, :, 0] - ps1[:, 0]) <= 1e-8 * np.abs(ps1[:, 0]))
    assert np.all(np.abs(ps[2, :, 0] - refs[2]["q"][:, 0]) <= 1e-4 * np.abs(refs[2]["q"][:, 0]))


def test_multi_plan_replay(Q):
    """A shared-lattice plan replays bit-identically."""
    probs = I.config3_shared(count=9, d=6, n=1000003, m=8)
    g = I.random_generating_vector(I.SplitMix64(65), 6, probs[0].n)
    fs = [Q.integrand_from_problem(p, "fp32") for p in probs]
    plan = Q.qmc_multi_plan_create(6, probs[0].n, 8, g, probs[0].shifts, Q.transform("baker"), fs)
    a = plan.execute()
    b = plan.execute()
    assert len(a) == 10
    assert all(x.mean[0] == y.mean[0] and x.err[0] == y.err[0] for x, y in zip(a, b))
    desc = plan.describe()
    assert desc["orders"] == "10" and desc["specialised"] == "1"
    assert plan.launches() == 4 * 2 + 1
    plan.destroy()


@pytest.mark.slow
def test_multi_full_size(Q, oracle_lib, nthreads):
    """The fused sweep at the size the benchmark times it (32 sectors, d = 6,
    n = 16777213, m = 16, baker): every integrand's per-shift values against
    the same integrands run one kernel each (a graph batch, 1e-8: the same
    per-point values, grouped differently), the sum group equal to the sum of
    the integrands, and two integrands' first two shifts against the oracle
    over all 16.7M points (2e-7)."""
    import dataclasses
    probs = I.config3_shared()
    n, m = probs[0].n, probs[0].m
    g = I.random_generating_vector(I.SplitMix64(64), 6, n)
    fs = [Q.integrand_from_problem(p, "fp32") for p in probs]
    t = Q.transform("baker")
    res, ps = Q.qmc_integrate_multi(6, n, m, g, probs[0].shifts, t, fs, want_per_shift=True)
    assert all(r.status == 0 for r in res)
    bp = Q.BatchPlan([(6, n, m, g, probs[0].shifts, t, f) for f in fs])
    ps_b = np.zeros(2 * m * len(fs))
    bp.execute(per_shift=ps_b)
    bp.destroy()
    ps_b = ps_b.reshape(len(fs), m, 2)
    assert np.all(np.abs(ps[:32, :, 0] - ps_b[:, :, 0]) <= 1e-8 * np.abs(ps_b[:, :, 0]))
    assert np.allclose(ps[32, :, 0], ps[:32, :, 0].sum(axis=0), rtol=1e-13, atol=0)
    for s in (0, 31):
        p2 = dataclasses.replace(probs[s], m=2, shifts=probs[s].shifts[:2].copy())
        ref = oracle_lib.integrate(p2, g, nthreads=nthreads)["q"][:, 0]
        assert np.all(np.abs(ps[s, :2, 0] - ref) <= 2e-7 * np.abs(ref)), s

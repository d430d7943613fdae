"""GPU parity of the epsilon expansion of Eq. (7): the coefficient integrands
f_k = U^aU F^aF L^k / k!, L = bU log U + bF log F, estimated for all orders
in one pass, against the oracle's per-order integrand.

Tolerances.  Order k's value carries the order-0 error plus k times the
error of L; |L| <= A with A = |bU| max|log U| + |bF| max|log F| over the
cube (bounded from the coefficient ranges: every coefficient of these inputs
is positive, so c0 <= P <= sum of coefficients).  So order k is compared
within (k + 1) tol |v_0| (A + 1)^k / k!, tol being the order-0 tolerance of
the plain path (1e-13 per point FP64, 4e-6 FP32; Q^(k) 1e-12 / 4e-7 of the
same scale)."""
import math
import os

import numpy as np
import pytest

from paper_1811_11722_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    from paper_1811_11722_gb300 import build, qmc
    build.build_library()
    return qmc


def log_bound(poly):
    """max |log P| over the unit cube for P with positive coefficients."""
    lo = float(poly.coef[np.all(poly.expo == 0, axis=1)].sum())
    hi = float(poly.coef.sum())
    return max(abs(math.log(lo)), abs(math.log(hi)))


def scale_k(k, A):
    return (k + 1) * (A + 1.0) ** k / math.factorial(k)


def eps_problem(p, orders, bU=1.0, bF=-1.0):
    p.eps = {"order": 0, "bU": bU, "bF": bF}
    return p


def oracle_orders(oracle_lib, p, g, orders, nthreads=1):
    out = []
    for o in range(orders):
        p.eps = dict(p.eps, order=o)
        out.append(oracle_lib.integrate(p, g, nthreads=nthreads))
    p.eps = dict(p.eps, order=0)
    return out


def sector(d, n, m, seed, transform="baker", alpha=0, n_lin=None, n_quad=None):
    rng = I.SplitMix64(seed)
    U = I.random_poly(rng, d, d if n_lin is None else n_lin, 0)
    F = I.random_poly(rng, d, 0, d * (d + 1) // 2 if n_quad is None else n_quad)
    p = I.Problem("eps", d, n, m, I.make_shifts(rng, m, d), transform, alpha=alpha, kind="sector", U=U, F=F)
    g = I.random_generating_vector(rng, d, n)
    return p, g


# ------------------------------------------------------------ single points --

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("transform,alpha", [("baker", 0), ("korobov", 3), ("none", 0), ("korobov", 2)])
@pytest.mark.parametrize("orders", [3, 6])
def test_eps_points_vs_oracle(Q, oracle_lib, precision, transform, alpha, orders):
    """Every order at sampled (j, k): the dense fast path (baker, Korobov 3)
    and the general kernel (none, Korobov 2), at the full C2 size."""
    p = I.config2(n=16777213, m=32)
    p.transform, p.alpha = transform, alpha
    eps_problem(p, orders)
    g = I.random_generating_vector(I.SplitMix64(31), p.d, p.n)
    rng = np.random.default_rng(11)
    js = np.concatenate([[0, 1, p.n - 1], rng.integers(0, p.n, 120)]).astype(np.uint64)
    ks = np.concatenate([[0, 31, 7], rng.integers(0, p.m, 120)]).astype(np.int32)
    eps = Q.eps_spec(orders, 1.0, -1.0)
    vals = Q.qmc_sample_points_eps(p.d, p.n, p.m, g, p.shifts, Q.transform(transform, alpha),
                                   Q.integrand_from_problem(p, precision), eps, js, ks)
    A = log_bound(p.U) + log_bound(p.F)
    ctol = 2.0 ** -52 if precision == "fp64" else 2.0 ** -23
    vtol = 1e-13 if precision == "fp64" else 4e-6
    for s in range(len(js)):
        ref = []
        for o in range(orders):
            p.eps["order"] = o
            v, _, ox, _, _ = oracle_lib.point(p, g, int(ks[s]), int(js[s]))
            ref.append(v[0])
        p.eps["order"] = 0
        rel = vtol
        if transform == "korobov":
            sdist = np.minimum(ox, 1.0 - ox)
            rel += float(np.sum(2 * alpha * ctol / np.maximum(sdist, 1e-300)))
        for o in range(orders):
            tol = rel * scale_k(o, A) * abs(ref[0]) + 1e-300
            assert abs(vals[s, o] - ref[o]) <= tol, (s, o, vals[s, o], ref[o])


# ------------------------------------------------------------- whole rule --

@pytest.mark.parametrize("transform,alpha", [("baker", 0), ("korobov", 3), ("none", 0)])
@pytest.mark.parametrize("orders", [1, 3, 5])
def test_eps_rule_fp64_vs_oracle(Q, oracle_lib, nthreads, transform, alpha, orders):
    """d=6 sector, n = 100003 (many tiles and a ragged tail), m = 10 (several
    shift chunks with padded rows): per-shift Q^(k) of every order."""
    p, g = sector(6, 100003, 10, 41, transform, alpha)
    eps_problem(p, orders)
    f = Q.integrand_from_problem(p, "fp64")
    res, ps = Q.qmc_integrate_eps(p.d, p.n, p.m, g, p.shifts, Q.transform(transform, alpha), f,
                                  Q.eps_spec(orders), want_per_shift=True)
    refs = oracle_orders(oracle_lib, p, g, orders, nthreads)
    A = log_bound(p.U) + log_bound(p.F)
    q0 = abs(refs[0]["mean"][0])
    for o in range(orders):
        tol = 1e-12 * scale_k(o, A) * q0
        assert res[o].status == 0 and res[o].nonfinite == 0
        assert np.all(np.abs(ps[o, :, 0] - refs[o]["q"][:, 0]) <= tol), o
        assert abs(res[o].mean[0] - refs[o]["mean"][0]) <= tol, o
        assert abs(res[o].err[0] - refs[o]["err"][0]) <= 2 * tol, o
        assert np.all(ps[o, :, 1] == 0.0)


@pytest.mark.parametrize("transform,alpha", [("baker", 0), ("korobov", 3)])
def test_eps_rule_fp32_vs_oracle(Q, oracle_lib, nthreads, transform, alpha):
    p, g = sector(6, 100003, 16, 42, transform, alpha)
    eps_problem(p, 4)
    f = Q.integrand_from_problem(p, "fp32")
    res, ps = Q.qmc_integrate_eps(p.d, p.n, p.m, g, p.shifts, Q.transform(transform, alpha), f,
                                  Q.eps_spec(4), want_per_shift=True)
    refs = oracle_orders(oracle_lib, p, g, 4, nthreads)
    A = log_bound(p.U) + log_bound(p.F)
    q0 = abs(refs[0]["mean"][0])
    for o in range(4):
        tol = 4e-7 * scale_k(o, A) * q0
        assert np.all(np.abs(ps[o, :, 0] - refs[o]["q"][:, 0]) <= tol), o
        assert abs(res[o].mean[0] - refs[o]["mean"][0]) <= tol, o


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 7, 8, 10])
def test_eps_all_dims(Q, oracle_lib, d):
    """Every specialised dimension (d <= 8) and the general kernel (d = 10)."""
    p, g = sector(d, 20011, 9, 200 + d, "korobov", 3)
    eps_problem(p, 3)
    f = Q.integrand_from_problem(p, "fp64")
    res, ps = Q.qmc_integrate_eps(p.d, p.n, p.m, g, p.shifts, Q.transform("korobov", 3), f, Q.eps_spec(3),
                                  want_per_shift=True)
    refs = oracle_orders(oracle_lib, p, g, 3)
    A = log_bound(p.U) + log_bound(p.F)
    q0 = abs(refs[0]["mean"][0])
    for o in range(3):
        assert np.all(np.abs(ps[o, :, 0] - refs[o]["q"][:, 0]) <= 1e-12 * scale_k(o, A) * q0), (d, o)


def test_eps_order0_is_the_plain_rule(Q):
    """Order 0 is the SECTOR integrand itself: same estimate as qmc_integrate."""
    p, g = sector(6, 100003, 12, 43, "baker")
    for prec, tol in (("fp64", 1e-13), ("fp32", 2e-7)):
        f = Q.integrand_from_problem(p, prec)
        t = Q.transform("baker")
        plain, ps_plain = Q.qmc_integrate(p.d, p.n, p.m, g, p.shifts, t, f, want_per_shift=True)
        res, ps = Q.qmc_integrate_eps(p.d, p.n, p.m, g, p.shifts, t, f, Q.eps_spec(2), want_per_shift=True)
        assert np.all(np.abs(ps[0, :, 0] - ps_plain[:, 0]) <= tol * np.abs(ps_plain[:, 0])), prec
        assert abs(res[0].mean[0] - plain.mean[0]) <= tol * abs(plain.mean[0])


def test_eps_slopes_general(Q, oracle_lib):
    """Other slopes and powers: U^(-3 + 2 eps) F^(-2 - 0.5 eps), which the dense
    fast path does not serve (general kernel)."""
    p, g = sector(4, 10007, 4, 44, "korobov", 3)
    p.aU, p.aF = -3, -2
    eps_problem(p, 4, 2.0, -0.5)
    f = Q.integrand_from_problem(p, "fp64")
    res, ps = Q.qmc_integrate_eps(p.d, p.n, p.m, g, p.shifts, Q.transform("korobov", 3), f,
                                  Q.eps_spec(4, 2.0, -0.5), want_per_shift=True)
    refs = oracle_orders(oracle_lib, p, g, 4)
    A = 2.0 * log_bound(p.U) + 0.5 * log_bound(p.F)
    q0 = abs(refs[0]["mean"][0])
    for o in range(4):
        assert np.all(np.abs(ps[o, :, 0] - refs[o]["q"][:, 0]) <= 1e-12 * scale_k(o, A) * q0), o


def test_eps_nonfinite_counted_per_order(Q, oracle_lib):
    """U = 0.3 - z_1 + ... changes sign on the cube: order 0 (U^-2) stays
    finite while log U is NaN for orders >= 1.  Each order counts its own
    non-finite values, as the oracle does."""
    d, n, m = 2, 1009, 3
    U = I.Poly(np.array([0.3, -1.0, 0.5]), np.array([[0, 0], [1, 0], [0, 1]], np.uint8))
    F = I.Poly(np.array([1.0, 1.0]), np.array([[0, 0], [1, 1]], np.uint8))
    rng = I.SplitMix64(45)
    p = I.Problem("nf", d, n, m, I.make_shifts(rng, m, d), "baker", kind="sector", U=U, F=F)
    eps_problem(p, 3)
    g = np.array([1, 17], dtype=np.uint64)
    f = Q.integrand_from_problem(p, "fp64")
    res, ps = Q.qmc_integrate_eps(d, n, m, g, p.shifts, Q.transform("baker"), f, Q.eps_spec(3),
                                  want_per_shift=True)
    refs = oracle_orders(oracle_lib, p, g, 3)
    assert int(refs[0]["nonfinite"].sum()) == 0 and res[0].nonfinite == 0 and res[0].status == 0
    for o in (1, 2):
        nf = int(refs[o]["nonfinite"].sum())
        assert nf > 0
        assert res[o].nonfinite == nf
        assert res[o].status == Q.QMC_ENONFINITE
        assert np.allclose(ps[o, :, 0], refs[o]["q"][:, 0], rtol=1e-12, atol=1e-14)


def test_eps_plan_reproducible_and_device_output(Q):
    """An epsilon plan replays bit-identically; device outputs match host ones."""
    import torch
    p, g = sector(6, 1000003, 16, 46, "baker")
    f = Q.integrand_from_problem(p, "fp32")
    plan = Q.qmc_eps_plan_create(p.d, p.n, p.m, g, p.shifts, Q.transform("baker"), f, Q.eps_spec(3))
    a = plan.execute()
    b = plan.execute()
    assert len(a) == 3
    for o in range(3):
        assert a[o].mean[0] == b[o].mean[0] and a[o].err[0] == b[o].err[0]
    out = torch.zeros(3 * Q.RESULT_BYTES // 8, dtype=torch.float64, device="cuda")
    ps = torch.zeros(3 * p.m * 2, dtype=torch.float64, device="cuda")
    plan.execute(out=out, per_shift=ps)
    torch.cuda.synchronize()
    host = out.cpu().numpy().reshape(3, Q.RESULT_BYTES // 8)
    for o in range(3):
        assert host[o, 0] == a[o].mean[0]
    assert plan.describe()["orders"] == "3"
    plan.destroy()

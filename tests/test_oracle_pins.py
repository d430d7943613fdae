"""Pins of the CPU oracle against facts that do not come from the oracle itself:
exact rational brute force, closed-form integrals, library routines
(scipy quad / betainc, numpy det / var, Gauss-Legendre), invariances the paper
states, and brute-force optimality of the generating-vector search.

Each pin is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign, index or normalisation, a transposed operand) fails at least one.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_1811_11722_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def small_sector(d, seed, transform="baker", alpha=0, n=1009, m=4, n_lin=None, n_quad=None,
                 kind="sector", lam=0.0, neg_quad=0):
    rng = I.SplitMix64(seed)
    U = I.random_poly(rng, d, d if n_lin is None else n_lin, 0)
    F = I.random_poly(rng, d, 0, (d * (d + 1)) // 2 if n_quad is None else n_quad, neg_quad=neg_quad)
    shifts = I.make_shifts(rng, m, d)
    return I.Problem(f"small_{d}_{seed}", d, n, m, shifts, transform, alpha=alpha, kind=kind,
                     U=U, F=F, aU=-2, aF=-1, lam=lam)


# ------------------------------------------------------------------ indices --

def test_index_exact_bigint(oracle_lib):
    """Eq. (2) index (j-1) g mod n against Python big integers, including products above 2^64."""
    rng = I.SplitMix64(1)
    for _ in range(2000):
        n = rng.randint(2, (1 << 40))
        g = rng.randint(1, n - 1)
        j = rng.randint(0, n - 1)
        assert oracle_lib.index(j, g, n) == (j * g) % n


# ------------------------------------------------- exact rational brute force --

def _korobov_exact(alpha):
    """Korobov z(x) and w(x) as exact rational polynomials from sympy's integral."""
    sympy = pytest.importorskip("sympy")
    u, x = sympy.symbols("u x")
    norm = sympy.integrate(u ** alpha * (1 - u) ** alpha, (u, 0, 1))
    w = sympy.Poly(sympy.expand(x ** alpha * (1 - x) ** alpha / norm), x)
    z = sympy.Poly(sympy.integrate(sympy.expand(u ** alpha * (1 - u) ** alpha / norm), (u, 0, x)), x)

    def ev(poly, t):
        acc = Fraction(0)
        for (k,), c in poly.terms():
            acc += Fraction(int(c.p), int(c.q)) * t ** k
        return acc
    return (lambda t: ev(z, t)), (lambda t: ev(w, t))


def _exact_rule(p, g, shifts_frac, transform, alpha):
    """Eq. (2)/(3) in exact rational arithmetic for a small lattice."""
    if transform == "korobov":
        zf, wf = _korobov_exact(alpha)
    qs = []
    for sh in shifts_frac:
        tot = Fraction(0)
        for j in range(p.n):
            z, w = [], Fraction(1)
            for i in range(p.d):
                y = Fraction((j * int(g[i])) % p.n, p.n) + sh[i]
                x = y - 1 if y >= 1 else y
                if transform == "baker":
                    z.append(1 - abs(2 * x - 1))
                elif transform == "korobov":
                    z.append(zf(x))
                    w *= wf(x)
                else:
                    z.append(x)
            U = Fraction(0)
            for c, e in zip(p.U.coef, p.U.expo):
                t = Fraction(c)
                for i in range(p.d):
                    t *= z[i] ** int(e[i])
                U += t
            F = Fraction(0)
            for c, e in zip(p.F.coef, p.F.expo):
                t = Fraction(c)
                for i in range(p.d):
                    t *= z[i] ** int(e[i])
                F += t
            tot += w * U ** p.aU * F ** p.aF
        qs.append(tot / p.n)
    m = len(qs)
    qbar = sum(qs) / m
    var = sum((q - qbar) ** 2 for q in qs) / (m * (m - 1))
    return qs, qbar, var


@pytest.mark.parametrize("transform,alpha,n,d", [("none", 0, 13, 2), ("baker", 0, 31, 2),
                                                  ("korobov", 3, 17, 2), ("baker", 0, 11, 3),
                                                  ("korobov", 2, 7, 3)])
def test_rule_matches_exact_rationals(oracle_lib, transform, alpha, n, d):
    """Whole rule (indices, fractional part, transform, U^-2 F^-1, sums, mean,
    variance) against exact rational arithmetic on tiny lattices with dyadic
    coefficients and shifts a/1024."""
    rng = I.SplitMix64(77 + n + d)
    m = 3
    p = small_sector(d, 5 + n, transform=transform, alpha=alpha, n=n, m=m)
    # dyadic coefficients so the double inputs are exact rationals
    p.U.coef[:] = np.round(p.U.coef * 64) / 64
    p.F.coef[:] = np.round(p.F.coef * 64) / 64
    shifts_frac = [[Fraction(rng.randint(0, 1023), 1024) for _ in range(d)] for _ in range(m)]
    p.shifts = np.array([[float(s) for s in row] for row in shifts_frac])
    g = np.array([1] + [rng.randint(1, n - 1) for _ in range(d - 1)], dtype=np.uint64)
    qs, qbar, var = _exact_rule(p, g, shifts_frac, transform, alpha)
    r = oracle_lib.integrate(p, g)
    for k in range(m):
        assert abs(r["q"][k, 0] - float(qs[k])) <= 8e-16 * abs(float(qs[k]))
    assert abs(r["mean"][0] - float(qbar)) <= 8e-16 * abs(float(qbar))
    assert abs(r["var"][0] - float(var)) <= 1e-10 * float(var) + 1e-30


# ------------------------------------------------------------ closed forms --

def test_constant_baker_is_exact(oracle_lib):
    """Sec. 2 / Fig. 3 text: baker on the constant 1 has zero error for any lattice."""
    gold = json.load(open(os.path.join(GOLDEN, "constant_integrand.json")))
    for d in gold["korobov_dimensions"]:
        rng = I.SplitMix64(d)
        n = 1021
        p = I.Problem("const", d, n, 5, I.make_shifts(rng, 5, d), "baker", kind="const")
        g = I.random_generating_vector(rng, d, n)
        r = oracle_lib.integrate(p, g)
        assert np.all(r["q"][:, 0] == gold["baker_per_shift_value"])
        assert r["var"][0] == gold["baker_variance"]


def test_constant_korobov_converges(oracle_lib):
    """Fig. 3: the constant 1 under Korobov 3 in d = 6 converges to 1 (error
    shrinks from n ~ 1e3 to n ~ 1e5) and the estimate brackets the error."""
    from oracle.cbc import cbc_fast
    d, alpha = 6, 3
    errs = []
    for n in (1021, 16381, 131071):
        g = cbc_fast(d, n, I.product_weights(d))
        rng = I.SplitMix64(11)
        p = I.Problem("const", d, n, 8, I.make_shifts(rng, 8, d), "korobov", alpha=alpha, kind="const")
        r = oracle_lib.integrate(p, g, nthreads=4)
        errs.append(abs(r["mean"][0] - 1.0))
        assert abs(r["mean"][0] - 1.0) < 6.0 * r["err"][0] + 1e-14
    assert errs[2] < errs[0] / 20


def test_separable_closed_form(oracle_lib):
    """Configuration 1 integrand prod (1 + c x) e^{b x}: the rule with Korobov 3
    approaches the closed form prod ((-b + c + (bc + b - c) e^b) / b^2)."""
    from oracle.cbc import cbc_fast
    p = I.config1(n=65521, m=10)
    exact = 1.0
    for c, b in zip(p.c, p.b):
        exact *= (-b + c + (b * c + b - c) * math.exp(b)) / (b * b)
    g = cbc_fast(p.d, p.n, p.gamma)
    r = oracle_lib.integrate(p, g, nthreads=4)
    assert abs(r["mean"][0] - exact) < 5 * r["err"][0] + 1e-14
    assert abs(r["mean"][0] - exact) < 1e-9 * exact


def test_sector_d1_against_quad(oracle_lib):
    """d = 1, U = a + b x, F = c + e x^2: the rule vs scipy's adaptive quadrature."""
    quad = pytest.importorskip("scipy.integrate").quad
    a, b, c, e = 0.7, 1.3, 0.4, 1.9
    U = I.Poly(np.array([a, b]), np.array([[0], [1]], dtype=np.uint8))
    F = I.Poly(np.array([c, e]), np.array([[0], [2]], dtype=np.uint8))
    ref, _ = quad(lambda x: 1.0 / ((a + b * x) ** 2 * (c + e * x * x)), 0, 1, epsabs=1e-15, epsrel=1e-14)
    rng = I.SplitMix64(3)
    p = I.Problem("d1", 1, 65521, 6, I.make_shifts(rng, 6, 1), "korobov", alpha=3, kind="sector", U=U, F=F)
    r = oracle_lib.integrate(p, [1])
    assert abs(r["mean"][0] - ref) < 1e-11 * ref
    gl = oracle_lib.gauss_legendre(p, 60)
    assert abs(gl[0] - ref) < 1e-13 * ref


def test_polynomial_integrand_exact_by_gauss_legendre(oracle_lib):
    """Positive powers make U^aU F^aF a polynomial; its integral over the cube is
    sum of coef * prod 1/(e_i + 1) per monomial of the expanded product, which
    tensor Gauss-Legendre with enough nodes reproduces exactly."""
    sympy = pytest.importorskip("sympy")
    d = 3
    p = small_sector(d, 19)
    p.aU, p.aF = 2, 1
    xs = sympy.symbols(f"x0:{d}")
    Ue = sum(sympy.Rational(float(c)) * sympy.prod([xs[i] ** int(e[i]) for i in range(d)])
             for c, e in zip(p.U.coef, p.U.expo))
    Fe = sum(sympy.Rational(float(c)) * sympy.prod([xs[i] ** int(e[i]) for i in range(d)])
             for c, e in zip(p.F.coef, p.F.expo))
    expr = sympy.expand(Ue ** 2 * Fe)
    exact = expr
    for x in xs:
        exact = sympy.integrate(exact, (x, 0, 1))
    gl = oracle_lib.gauss_legendre(p, 4)
    assert abs(gl[0] - float(exact)) < 1e-13 * abs(float(exact))


def test_sector_rule_vs_gauss_legendre(oracle_lib):
    """A d = 4 sector integrand (analytic on the closed cube): the baker rule at
    n ~ 1.3e5 against tensor Gauss-Legendre, which has itself converged."""
    from oracle.cbc import cbc_fast
    p = small_sector(4, 23, transform="baker", n=131071, m=8, n_quad=6)
    gl16 = oracle_lib.gauss_legendre(p, 16, nthreads=4)
    gl20 = oracle_lib.gauss_legendre(p, 20, nthreads=4)
    assert abs(gl16[0] - gl20[0]) < 1e-13 * abs(gl20[0])
    g = cbc_fast(p.d, p.n, I.product_weights(p.d))
    r = oracle_lib.integrate(p, g, nthreads=4)
    assert abs(r["mean"][0] - gl20[0]) < 5 * r["err"][0] + 1e-13


def test_transform_invariance(oracle_lib):
    """The integral does not depend on the periodizing transform (Eq. 5, 6):
    none, baker, Korobov 3 and Korobov 6 agree within the combined error."""
    from oracle.cbc import cbc_fast
    n = 65521
    g = cbc_fast(3, n, I.product_weights(3))
    base = small_sector(3, 29, n=n, m=10)
    gl = oracle_lib.gauss_legendre(base, 24)[0]
    for tr, al in (("none", 0), ("baker", 0), ("korobov", 3), ("korobov", 6)):
        p = small_sector(3, 29, transform=tr, alpha=al, n=n, m=10)
        r = oracle_lib.integrate(p, g, nthreads=4)
        tol = 6 * r["err"][0] + 1e-13
        assert abs(r["mean"][0] - gl) < tol, (tr, al, r["mean"][0], gl, r["err"][0])


# -------------------------------------------------------------- transforms --

@pytest.mark.parametrize("alpha", [1, 2, 3, 4, 5, 6])
def test_korobov_transform(oracle_lib, alpha):
    """Eq. (5): z is the regularized incomplete beta I_x(a+1, a+1) (scipy), the
    weight integrates to 1 and equals dz/dx."""
    betainc = pytest.importorskip("scipy.special").betainc
    xs = np.linspace(0.0, 1.0, 257)
    for x in xs:
        z, w = oracle_lib.transform("korobov", alpha, x)
        assert abs(z - betainc(alpha + 1, alpha + 1, x)) < 1e-14
    # integral of the weight by Gauss-Legendre with alpha+1 nodes (exact, degree 2 alpha)
    t, wt = np.polynomial.legendre.leggauss(alpha + 1)
    s = sum(0.5 * wi * oracle_lib.transform("korobov", alpha, 0.5 * (ti + 1))[1] for ti, wi in zip(t, wt))
    assert abs(s - 1.0) < 1e-14
    h = 1e-5
    for x in (0.1, 0.37, 0.5, 0.81):
        zp = oracle_lib.transform("korobov", alpha, x + h)[0]
        zm = oracle_lib.transform("korobov", alpha, x - h)[0]
        w = oracle_lib.transform("korobov", alpha, x)[1]
        assert abs((zp - zm) / (2 * h) - w) < 1e-8 * max(1.0, w)


def test_baker_transform(oracle_lib):
    """Eq. (6): z = 1 - |2x - 1|, piecewise slope +-2, weight 1; it maps both
    halves onto [0, 1], so int f(z(x)) dx = int f (here 1 + 3 z^2 -> 2)."""
    quad = pytest.importorskip("scipy.integrate").quad
    for x, zexp in ((0.0, 0.0), (0.25, 0.5), (0.5, 1.0), (0.75, 0.5), (1.0, 0.0)):
        z, w = oracle_lib.transform("baker", 0, x)
        assert z == zexp and w == 1.0
    val, _ = quad(lambda x: 1 + 3 * oracle_lib.transform("baker", 0, x)[0] ** 2, 0, 1, points=[0.5])
    assert abs(val - 2.0) < 1e-13


# --------------------------------------------------------------- estimator --

def test_variance_estimate(oracle_lib):
    """Eq. (3): with m = 2, sigma^2 = (Q1 - Q2)^2 / 4; in general it equals
    numpy's unbiased sample variance divided by m."""
    sums = np.array([[3.0, 0.5], [5.0, -0.5]])
    q, mean, var = oracle_lib.estimate(sums, 2)
    assert mean[0] == 2.0 and var[0] == ((1.5 - 2.5) ** 2) / 4
    assert mean[1] == 0.0 and var[1] == ((0.25 + 0.25) ** 2) / 4
    rng = np.random.default_rng(5)
    s = rng.normal(size=(17, 2))
    q, mean, var = oracle_lib.estimate(s, 7)
    assert np.allclose(mean, (s / 7).mean(axis=0), rtol=1e-15, atol=0)
    assert np.allclose(var, (s / 7).var(axis=0, ddof=1) / 17, rtol=1e-13, atol=0)
    with pytest.raises(ValueError):
        oracle_lib.estimate(s[:1], 7)


def test_shift_rule_unbiased(oracle_lib):
    """Eq. (2): each randomly shifted rule is an unbiased estimate.  Over 200
    independent shift tables the mean of Qbar - I is within 4 standard errors."""
    p0 = I.config1(n=1021, m=4)
    exact = 1.0
    for c, b in zip(p0.c, p0.b):
        exact *= (-b + c + (b * c + b - c) * math.exp(b)) / (b * b)
    g = oracle_lib.cbc_plain(3, 1021, p0.gamma)
    p0 = I.Problem(p0.name, 3, 1021, 4, p0.shifts, "none", kind="separable_exp", c=p0.c, b=p0.b)
    devs = []
    for s in range(200):
        p = I.with_shifts(p0, 4, 1000 + s)
        r = oracle_lib.integrate(p, g)
        devs.append(r["mean"][0] - exact)
    devs = np.array(devs)
    assert abs(devs.mean()) < 4 * devs.std(ddof=1) / math.sqrt(len(devs))


def test_dual_lattice_exactness(oracle_lib):
    """Eq. (2) on f = cos(2 pi h.x) without transform: Q^(k) = cos(2 pi h.Delta_k)
    if h.g = 0 mod n (h in the dual lattice) and 0 otherwise."""
    n, g = 101, np.array([1, 39, 17], dtype=np.uint64)
    rng = I.SplitMix64(9)
    sh = I.make_shifts(rng, 4, 3)
    for h in ([-39, 1, 0], [17, 0, -1], [1, 1, 0], [3, -2, 5], [0, 0, 0]):
        h = np.array(h, dtype=np.int32)
        p = I.Problem("trig", 3, n, 4, sh, "none", kind="trig", h=h)
        r = oracle_lib.integrate(p, g)
        dual = int(np.dot(h.astype(np.int64), g.astype(np.int64))) % n == 0
        for k in range(4):
            want = math.cos(2 * math.pi * float(np.dot(h, sh[k]))) if dual else 0.0
            assert abs(r["q"][k, 0] - want) < 1e-13


# ---------------------------------------------------------------- integrand --

def test_zbb_F_vanishes(oracle_lib):
    """Eq. (11): F/m_Z^2 vanishes at x0=x1=x2=x4=x5=1, x3=1/2; along that line
    (x3 = t) it is the quadratic 4t^2 + 6t - 4 (sympy expansion of the table)."""
    sympy = pytest.importorskip("sympy")
    gold = json.load(open(os.path.join(GOLDEN, "zbb_vertex.json")))
    F = I.zbb_vertex_F()
    assert F.degree == gold["degree"]
    assert int((F.coef > 0).sum()) == gold["signs"]["positive_terms"]
    assert int((F.coef < 0).sum()) == gold["signs"]["negative_terms"]
    one = I.Poly(np.array([1.0]), np.zeros((1, 6), dtype=np.uint8))
    p = I.Problem("zbb", 6, 2, 2, np.zeros((2, 6)), "none", kind="sector", U=one, F=F, aU=0, aF=1)
    v, _ = oracle_lib.integrand(p, gold["point"])
    assert v[0] == gold["F_at_point"]
    t = sympy.symbols("t")
    xs = [1, 1, 1, t, 1, 1]
    line = sympy.expand(sum(int(c) * sympy.prod([xs[i] ** int(e[i]) for i in range(6)])
                            for c, e in zip(F.coef, F.expo)))
    for tv in (0.0, 0.2, 0.7, 1.0):
        v, _ = oracle_lib.integrand(p, [1, 1, 1, tv, 1, 1])
        assert abs(v[0] - float(line.subs(t, tv))) < 1e-14


def test_det_lu_against_numpy(oracle_lib):
    """LU with partial pivoting vs numpy.linalg.det, including a zero leading pivot."""
    rng = np.random.default_rng(0)
    for d in (1, 2, 3, 5, 8):
        a = rng.normal(size=(d, d)) + 1j * rng.normal(size=(d, d))
        assert abs(oracle_lib.det_lu(a) - np.linalg.det(a)) < 1e-12 * max(1.0, abs(np.linalg.det(a)))
    a = np.array([[0, 1, 2], [3, 0, 1], [1, 1, 0]], dtype=complex)
    assert abs(oracle_lib.det_lu(a) - np.linalg.det(a)) < 1e-13


def test_deformation_at_corners(oracle_lib):
    """Sec. 3: the deformation vanishes at the endpoints, so at a corner of the
    cube z = y and J is diagonal with J_kk = 1 - i lam (1 - 2 y_k) dF/dy_k:
    the deformed value is the undeformed U^-2 F^-1 times that product."""
    p = small_sector(3, 31, kind="sector_deformed", lam=0.1, transform="none", neg_quad=2)
    q = small_sector(3, 31, kind="sector", transform="none", neg_quad=2)
    sympy = pytest.importorskip("sympy")
    xs = sympy.symbols("x0:3")
    Fe = sum(sympy.Rational(float(c)) * sympy.prod([xs[i] ** int(e[i]) for i in range(3)])
             for c, e in zip(p.F.coef, p.F.expo))
    for corner in ([0, 0, 0], [1, 0, 1], [1, 1, 1], [0, 1, 0]):
        v, _ = oracle_lib.integrand(p, corner)
        u, _ = oracle_lib.integrand(q, corner)
        det = 1.0 + 0j
        for k in range(3):
            dF = float(sympy.diff(Fe, xs[k]).subs(dict(zip(xs, corner))))
            det *= 1 - 1j * 0.1 * (1 - 2 * corner[k]) * dF
        want = u[0] * det
        assert abs(complex(v[0], v[1]) - want) < 1e-13 * abs(want)


def test_deformation_lambda_invariance(oracle_lib):
    """Cauchy's theorem: while no singularity is crossed the deformed integral
    does not depend on lambda (Gauss-Legendre, analytic integrand); for a
    positive F, lambda = 0 gives the same value."""
    pos = small_sector(3, 37, kind="sector_deformed", lam=0.1, transform="none")
    v1 = oracle_lib.gauss_legendre(pos, 24)
    pos.lam = 0.0
    v0 = oracle_lib.gauss_legendre(pos, 24)
    assert abs(v1[0] - v0[0]) < 1e-12 * abs(v0[0]) and abs(v1[1]) < 1e-12 * abs(v0[0])
    neg = small_sector(3, 41, kind="sector_deformed", lam=0.1, transform="none", neg_quad=2)
    a = oracle_lib.gauss_legendre(neg, 32)
    neg.lam = 0.05
    b = oracle_lib.gauss_legendre(neg, 32)
    assert abs(complex(*a) - complex(*b)) < 1e-8 * abs(complex(*a))


# --------------------------------------------------------------------- CBC --

def test_cbc_d1_closed_form(oracle_lib):
    """e^2 for d = 1, g = 1: gamma (1/n) sum_k B2(k/n) = gamma / (6 n^2)."""
    for n in (7, 31, 1009):
        assert abs(oracle_lib.cbc_error(1, n, [1], [0.5]) - 0.5 / (6 * n * n)) < 1e-15


@pytest.mark.parametrize("n", [7, 11, 13, 31])
def test_cbc_bruteforce(oracle_lib, n):
    """With g_1 = 1 the second CBC component is the global minimiser over all
    g_2 (brute force); in d = 3 the CBC error is >= the brute-force minimum and
    within a small factor of it."""
    gam = I.product_weights(3)
    g = oracle_lib.cbc_plain(3, n, gam)
    e2_2 = oracle_lib.cbc_error(2, n, g[:2], gam)
    brute2 = min(oracle_lib.cbc_error(2, n, [1, z], gam) for z in range(1, n))
    assert abs(e2_2 - brute2) <= 1e-15
    e3 = oracle_lib.cbc_error(3, n, g, gam)
    brute3 = min(oracle_lib.cbc_error(3, n, [1, a, b], gam) for a in range(1, n) for b in range(1, n))
    assert e3 >= brute3 - 1e-16 and e3 <= 1.5 * brute3


def test_cbc_fast_matches_plain(oracle_lib):
    """The convolution form of the search picks the same components as the
    plain O(n^2) search."""
    from oracle.cbc import cbc_fast
    gam = I.product_weights(8)
    for n in (31, 101, 1009, 4093, 10007):
        assert np.array_equal(cbc_fast(8 if n < 5000 else 4, n, gam), oracle_lib.cbc_plain(8 if n < 5000 else 4, n, gam))


# --------------------------------------------------------- control variate --

def test_cv_integral_closed_form(oracle_lib):
    """int g = sum_r prod_i a_ri0 against tensor Gauss-Legendre of g itself
    (g is a trigonometric polynomial of degree 31; 48 nodes per axis are exact
    to double precision)."""
    rng = np.random.default_rng(1)
    d, R, K = 2, 3, 8
    for F in (1, 2):
        a = rng.normal(size=R * d * K).astype(np.float32)
        x, w = np.polynomial.legendre.leggauss(48)
        x, w = 0.5 * (x + 1), 0.5 * w
        gl = sum(wi * wj * oracle_lib.cv_g(d, R, K, F, a, [xi, xj]) for xi, wi in zip(x, w) for xj, wj in zip(x, w))
        assert abs(gl - oracle_lib.cv_integral(d, R, K, a)) < 1e-12 * max(1.0, abs(gl))


def test_cv_gradient_finite_differences(oracle_lib):
    """The analytic FP64 gradient of the fit loss against central differences."""
    rng = np.random.default_rng(2)
    d, R, K, P = 3, 2, 6, 40
    a = (rng.normal(size=R * d * K) * 0.5).astype(np.float32)
    x = rng.random((P, d))
    h = rng.random(P)
    _, grad = oracle_lib.cv_loss_grad(d, R, K, 1, x, h, a)
    for q in rng.choice(R * d * K, 12, replace=False):
        ap, am = a.copy(), a.copy()
        ap[q] += np.float32(2.0 ** -8)
        am[q] -= np.float32(2.0 ** -8)
        lp, _ = oracle_lib.cv_loss_grad(d, R, K, 1, x, h, ap)
        lm, _ = oracle_lib.cv_loss_grad(d, R, K, 1, x, h, am)
        fd = (lp - lm) / (float(ap[q]) - float(am[q]))
        assert abs(fd - grad[q]) < 1e-4 * max(1.0, abs(grad[q]))


def test_cv_estimator_zero_surrogate_is_plain_rule(oracle_lib):
    """With a = 0 the control-variate estimate is the plain rule."""
    p = small_sector(3, 61, transform="korobov", alpha=3, n=2003, m=3)
    g = I.random_generating_vector(I.SplitMix64(61), 3, p.n)
    plain = oracle_lib.integrate(p, g)
    p.cv = {"R": 2, "K": 4, "F": 1, "a": np.zeros(2 * 3 * 4, np.float32)}
    cv = oracle_lib.integrate(p, g)
    assert np.array_equal(plain["q"], cv["q"])


def _cv_exact_surrogate(d, R, K, F, axis, freq):
    """Parameters whose rank 0 is cos(F pi k z_axis) with F k = 2 freq (so it
    equals cos(2 pi freq z_axis), the trig integrand with h = freq e_axis) and
    whose other ranks are zero."""
    a = np.zeros((R, d, K), np.float32)
    assert (2 * freq) % F == 0 and 2 * freq // F < K
    for i in range(d):
        a[0, i, 0] = 1.0
    a[0, axis, 0] = 0.0
    a[0, axis, 2 * freq // F] = 1.0
    return a.ravel()


@pytest.mark.parametrize("transform,alpha", [("none", 0), ("baker", 0), ("korobov", 3), ("korobov", 5)])
@pytest.mark.parametrize("F", [1, 2])
def test_cv_surrogate_equal_to_integrand_cancels(oracle_lib, transform, alpha, F):
    """With g = f the summand (f - g)(z(x)) prod w vanishes at every point, so
    every per-shift Q[f - g] is zero (to rounding) and the estimator returns
    int g = int f = 0 with zero variance.  f = cos(2 pi h.z) with h = 13 e_1
    on the n = 13 lattice: h is in the dual lattice (h.g = 13 = 0 mod 13), so
    without a transform the plain rule gives cos(2 pi h.Delta_k), far from 0
    (a sign slip in the subtraction doubles it).  Evaluating g at x instead of
    z, or leaving out the transform weight, leaves a Korobov-weighted
    cosine integral of order 0.1 per shift."""
    d, R, K, n, m, freq = 3, 2, 32, 13, 4, 13
    rng = I.SplitMix64(401 + F)
    h = np.zeros(d, np.int32)
    h[1] = freq
    p = I.Problem("trig_cv", d, n, m, I.make_shifts(rng, m, d), transform, alpha=alpha, kind="trig", h=h)
    g = np.array([1, 1, 5], dtype=np.uint64)
    plain = oracle_lib.integrate(p, g)
    if transform == "none":
        for k in range(m):
            assert abs(plain["q"][k, 0] - math.cos(2 * math.pi * freq * p.shifts[k, 1])) < 1e-12
    p.cv = {"R": R, "K": K, "F": F, "a": _cv_exact_surrogate(d, R, K, F, 1, freq)}
    assert oracle_lib.cv_integral(d, R, K, p.cv["a"]) == 0.0
    r = oracle_lib.integrate(p, g)
    assert np.all(np.abs(r["q"][:, 0]) < 1e-13), r["q"][:, 0]
    assert r["var"][0] < 1e-26


def _cv_generic_params(d, R, K, seed):
    """Surrogate parameters of the integrand's scale: constant terms near 0.8
    (so int g ~ R 0.8^d is not small), the rest N(0, 0.05)."""
    rng = np.random.default_rng(seed)
    a = rng.normal(0.0, 0.05, size=(R, d, K))
    a[:, :, 0] = 0.7 + 0.2 * rng.random((R, d))
    return a.astype(np.float32).ravel()


@pytest.mark.parametrize("transform,alpha", [("baker", 0), ("korobov", 3)])
@pytest.mark.parametrize("F", [1, 2])
def test_cv_estimator_unbiased_with_nonzero_surrogate(oracle_lib, transform, alpha, F):
    """Q[f - g] + int g estimates int f for any g (the shift average of the
    rule is unbiased for every integrable summand): a d = 3 sector integrand
    with a rank-2, K = 4 surrogate whose int g is about 1 agrees with tensor
    Gauss-Legendre of f within six Eq. (3) error estimates, under baker and
    Korobov 3.  Evaluating g at x instead of z (Korobov), dropping the weight
    from the g term (Korobov), or adding g instead of subtracting it moves the
    estimate by O(0.1)-O(1), far outside the error."""
    from oracle.cbc import cbc_fast
    d, R, K, n, m = 3, 2, 4, 32749, 8
    p = small_sector(d, 71, transform=transform, alpha=alpha, n=n, m=m)
    gl = oracle_lib.gauss_legendre(p, 24)[0]
    g = cbc_fast(d, n, I.product_weights(d))
    a = _cv_generic_params(d, R, K, seed=72 + F)
    gint = oracle_lib.cv_integral(d, R, K, a)
    assert 0.5 < gint < 2.0
    p.cv = {"R": R, "K": K, "F": F, "a": a}
    r = oracle_lib.integrate(p, g, nthreads=4)
    est = r["mean"][0] + gint
    assert abs(est - gl) < 6 * r["err"][0] + 1e-12, (est, gl, r["err"][0])
    # the surrogate term is live: every shift's Q[f - g] differs from Q[f] by about int g
    plain = oracle_lib.integrate(small_sector(d, 71, transform=transform, alpha=alpha, n=n, m=m), g, nthreads=4)
    assert np.all(np.abs(plain["q"][:, 0] - r["q"][:, 0]) > 0.5 * gint)


# ------------------------------------------------------- non-finite values --

def _exact_value(p, g, shift, j, zf, wf):
    """Term j of Eq. (2) in exact rationals for U = c0 + c1 z_0, F = z_1 (no
    constant, so F = 0 where x_1 = 0): returns None where F = 0 (the value is
    infinite, or 0 x infinite under Korobov), else the exact weighted value."""
    xs = []
    for i in range(p.d):
        y = Fraction((j * int(g[i])) % p.n, p.n) + Fraction(shift[i])
        xs.append(y - 1 if y >= 1 else y)
    z = [zf(x) for x in xs]
    w = Fraction(1)
    for x in xs:
        w *= wf(x)
    Fv = Fraction(p.F.coef[0]) * z[1]
    if Fv == 0:
        return None
    Uv = Fraction(p.U.coef[0]) + Fraction(p.U.coef[1]) * z[0]
    return w / (Uv * Uv * Fv)


@pytest.mark.parametrize("transform,alpha", [("none", 0), ("korobov", 3)])
def test_nonfinite_values_counted_and_left_out(oracle_lib, transform, alpha):
    """Reading R10 (points with a non-finite value are counted per shift and
    left out of the sum): on the n = 16 lattice with g = (1, 4), F = z_1 has
    no constant term and vanishes wherever x_1 = {4j/16 + Delta_1} = 0.  The
    count per shift equals a brute-force count in exact rationals (4, 4 and 0
    for the three dyadic shifts), and each per-shift sum equals the exact sum
    of the remaining terms.  Without a transform the value there is +inf;
    under Korobov 3 the weight is 0 too, and 0 x inf is NaN."""
    d, n = 2, 16
    g = np.array([1, 4], dtype=np.uint64)
    shifts = np.array([[0.125, 0.25], [0.5, 0.0], [0.3125, 0.0625]])
    U = I.Poly(np.array([0.75, 1.25]), np.array([[0, 0], [1, 0]], dtype=np.uint8))
    F = I.Poly(np.array([1.5]), np.array([[0, 1]], dtype=np.uint8))
    p = I.Problem("nonfinite", d, n, 3, shifts, transform, alpha=alpha, kind="sector", U=U, F=F, aU=-2, aF=-1)
    if transform == "korobov":
        zf, wf = _korobov_exact(alpha)
    else:
        zf, wf = (lambda t: t), (lambda t: Fraction(1))
    sums, nonf, _ = oracle_lib.rule_sums(p, g)
    want_counts = []
    for k in range(p.m):
        vals = [_exact_value(p, g, shifts[k], j, zf, wf) for j in range(n)]
        want_counts.append(sum(v is None for v in vals))
        exact = sum((v for v in vals if v is not None), Fraction(0))
        assert np.isfinite(sums[k, 0])
        assert abs(sums[k, 0] - float(exact)) <= 1e-14 * abs(float(exact)), (k, sums[k, 0], float(exact))
    assert want_counts == [4, 4, 0]
    assert [int(c) for c in nonf] == want_counts


# -------------------------------------------------------- epsilon expansion --

def test_eps_expansion_d1_against_quad(oracle_lib):
    """Eq. (7) with regulated powers: sum_k eps^k I_k of the coefficient
    integrands U^-2 F^-1 (bU log U + bF log F)^k / k! reproduces the integral
    of U^(-2 + bU eps) F^(-1 + bF eps) at small eps (scipy quad), and each I_k
    matches quad of its own coefficient integrand."""
    quad = pytest.importorskip("scipy.integrate").quad
    a, b, c, e = 0.7, 1.3, 0.4, 1.9
    bU, bF, eps = 1.0, -1.0, 0.05
    U = I.Poly(np.array([a, b]), np.array([[0], [1]], dtype=np.uint8))
    F = I.Poly(np.array([c, e]), np.array([[0], [2]], dtype=np.uint8))
    rng = I.SplitMix64(8)
    p = I.Problem("eps", 1, 65521, 6, I.make_shifts(rng, 6, 1), "korobov", alpha=3, kind="sector", U=U, F=F)
    total = 0.0
    for k in range(5):
        p.eps = {"order": k, "bU": bU, "bF": bF}
        r = oracle_lib.integrate(p, [1])
        ref_k, _ = quad(lambda x: (a + b * x) ** -2 * (c + e * x * x) ** -1
                        * (bU * math.log(a + b * x) + bF * math.log(c + e * x * x)) ** k / math.factorial(k),
                        0, 1, epsabs=1e-15, epsrel=1e-13)
        assert abs(r["mean"][0] - ref_k) < 1e-10 * max(1.0, abs(ref_k))
        total += eps ** k * r["mean"][0]
    full, _ = quad(lambda x: (a + b * x) ** (-2 + bU * eps) * (c + e * x * x) ** (-1 + bF * eps), 0, 1,
                   epsabs=1e-15, epsrel=1e-13)
    assert abs(total - full) < 2 * eps ** 5 * 10 + 1e-10


# ------------------------------------------- BF16 operands of the fit --

def test_bf16_rounding_matches_torch(oracle_lib):
    """The oracle's bfloat16 rounding (float first, then nearest-even to 8
    mantissa bits) against torch's float32 -> bfloat16 conversion."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(5)
    v = np.concatenate([rng.normal(size=2000) * 10.0 ** rng.integers(-8, 8, 2000),
                        [0.0, -0.0, 1.0, -1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 65504.0, 1e-30]])
    ref = torch.tensor(v.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([oracle_lib.bf16(x) for x in v])
    assert np.array_equal(got, ref)


def test_cv_fit_bf16_exact_operands(oracle_lib):
    """With operands that bfloat16 holds exactly (parameters on a 1/64 grid,
    points where every cos(pi k x) is 0, +-1/2 or +-1) the BF16 fit has the FP64
    fit's loss; its gradient differs only by the rounding of the factor
    2 e prod C / P, at most 2^-8 relative per term."""
    rng = np.random.default_rng(6)
    d, R, K, P = 3, 16, 32, 40
    a = (rng.integers(-32, 33, R * d * K) / 64.0).astype(np.float32)
    x = rng.choice([0.0, 0.5, 1.0 / 3.0, 2.0 / 3.0, 1.0], size=(P, d))
    h = rng.random(P)
    l64, g64 = oracle_lib.cv_loss_grad(d, R, K, 1, x, h, a)
    l16, g16 = oracle_lib.cv_loss_grad_bf16(d, R, K, 1, x, h, a)
    assert abs(l16 - l64) <= 1e-12 * l64
    # bound each gradient entry by the sum of |terms| (FP64 fit with |a|, |cos|, |e| is an upper bound proxy)
    assert np.max(np.abs(g16 - g64)) <= 2.0 ** -8 * np.max(np.abs(g64)) * 4
    # the factor's rounding does act, at BF16's scale (not just the last bits of a double)
    assert np.max(np.abs(g16 - g64)) > 1e-5 * np.max(np.abs(g64))


def test_cv_fit_bf16_close_to_fp64(oracle_lib):
    """For generic points the BF16 fit stays within BF16's resolution of the
    FP64 fit (loss within 2%, gradient within 2% of its largest entry)."""
    rng = np.random.default_rng(7)
    d, R, K, P = 4, 16, 32, 200
    a = (rng.normal(size=R * d * K) * 0.05).astype(np.float32)
    a[[(r * d + i) * K for r in range(R) for i in range(d)]] = 0.8
    x = rng.random((P, d))
    h = rng.random(P)
    l64, g64 = oracle_lib.cv_loss_grad(d, R, K, 1, x, h, a)
    l16, g16 = oracle_lib.cv_loss_grad_bf16(d, R, K, 1, x, h, a)
    assert abs(l16 - l64) <= 2e-2 * l64
    assert np.max(np.abs(g16 - g64)) <= 2e-2 * np.max(np.abs(g64))

"""Planted mistakes: each test copies oracle.c, plants one plausible slip (a
dropped term, a wrong sign, index, normalisation or denominator, a swapped
operand), builds the copy on the CPU, points the oracle's wrappers at it and
checks that at least one of the pins in test_oracle_pins.py now fails."""
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")

MUTATIONS = {
    "baker_sign": ("return 1.0 - fabs(2.0 * x - 1.0);", "return 1.0 - fabs(2.0 * x + 1.0);",
                   [pins.test_baker_transform]),
    "korobov_norm": ("return num / (den * den);", "return num / den;",
                     [lambda o: pins.test_korobov_transform(o, 3)]),
    "index_modulus": ("% (unsigned __int128)n);", "% (unsigned __int128)(n + 1));",
                      [pins.test_index_exact_bigint]),
    "no_wrap": ("x[i] = (y >= 1.0) ? y - 1.0 : y;", "x[i] = y;",
                [lambda o: pins.test_rule_matches_exact_rationals(o, "none", 0, 13, 2)]),
    "variance_denominator": ("var[part] = neum_get(&v) / ((double)m * (double)(m - 1));",
                             "var[part] = neum_get(&v) / ((double)m * (double)m);", [pins.test_variance_estimate]),
    "dropped_power": ("for (int q = 0; q < e[t * d + i]; ++q) p *= y[i];",
                      "for (int q = 1; q < e[t * d + i]; ++q) p *= y[i];",
                      [pins.test_polynomial_integrand_exact_by_gauss_legendre, pins.test_sector_d1_against_quad]),
    "weight_dropped": ("val[0] = f[0] * wprod;", "val[0] = f[0];", [pins.test_transform_invariance]),
    "shift_index": ("double y = (double)idx / (double)n + shift[i];", "double y = (double)idx / (double)n + shift[0];",
                    [lambda o: pins.test_rule_matches_exact_rationals(o, "baker", 0, 31, 2)]),
    "bernoulli_sign": ("static double bern2(double t) { return t * t - t + 1.0 / 6.0; }",
                       "static double bern2(double t) { return t * t + t + 1.0 / 6.0; }", [pins.test_cbc_d1_closed_form]),
    "jacobian_diagonal": ("im = -lam * (((k == l) ? (1.0 - 2.0 * y[k]) * grad[k] : 0.0) + y[k] * (1.0 - y[k]) * h2);",
                          "im = -lam * (((k == l) ? (1.0 - y[k]) * grad[k] : 0.0) + y[k] * (1.0 - y[k]) * h2);",
                          [pins.test_deformation_lambda_invariance, pins.test_deformation_at_corners]),
    "cv_integral_term": ("for (int i = 0; i < d; ++i) p *= (double)a[(r * d + i) * K];",
                         "for (int i = 1; i < d; ++i) p *= (double)a[(r * d + i) * K];", [pins.test_cv_integral_closed_form]),
    "bf16_ties_away": ("u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;", "u = (u + 0x8000u) & 0xFFFF0000u;",
                       [pins.test_bf16_rounding_matches_torch]),
    "bf16_factor_unrounded": ("const double dg = orc_bf16(2.0 * e * other / (double)P);",
                              "const double dg = 2.0 * e * other / (double)P;", [pins.test_cv_fit_bf16_exact_operands]),
    "cv_g_at_x": ("val[0] -= orc_cv_g(p->d, p->cvR, p->cvK, p->cvF, p->cva, z) * wprod;",
                  "val[0] -= orc_cv_g(p->d, p->cvR, p->cvK, p->cvF, p->cva, x) * wprod;",
                  [lambda o: pins.test_cv_surrogate_equal_to_integrand_cancels(o, "korobov", 3, 1),
                   lambda o: pins.test_cv_estimator_unbiased_with_nonzero_surrogate(o, "korobov", 3, 1)]),
    "cv_weight_dropped": ("val[0] -= orc_cv_g(p->d, p->cvR, p->cvK, p->cvF, p->cva, z) * wprod;",
                          "val[0] -= orc_cv_g(p->d, p->cvR, p->cvK, p->cvF, p->cva, z);",
                          [lambda o: pins.test_cv_surrogate_equal_to_integrand_cancels(o, "korobov", 3, 2),
                           lambda o: pins.test_cv_estimator_unbiased_with_nonzero_surrogate(o, "korobov", 3, 2)]),
    "cv_sign": ("val[0] -= orc_cv_g(", "val[0] += orc_cv_g(",
                [lambda o: pins.test_cv_surrogate_equal_to_integrand_cancels(o, "none", 0, 1),
                 lambda o: pins.test_cv_estimator_unbiased_with_nonzero_surrogate(o, "baker", 0, 1)]),
    "cv_basis_frequency": ("cos((double)F * M_PI * (double)k * x[i]);", "cos(M_PI * (double)k * x[i]);",
                           [lambda o: pins.test_cv_surrogate_equal_to_integrand_cancels(o, "baker", 0, 2)]),
    "nonfinite_not_counted": ("c->nonfinite[k] += 1;", "c->nonfinite[k] += 0;",
                              [lambda o: pins.test_nonfinite_values_counted_and_left_out(o, "none", 0)]),
    "nonfinite_summed": ("c->nonfinite[k] += 1;\n        continue;", "c->nonfinite[k] += 1;",
                         [lambda o: pins.test_nonfinite_values_counted_and_left_out(o, "korobov", 3)]),
    "eps_factorial_dropped": ("for (int k = 1; k <= p->eps_order; ++k) c *= L / (double)k;",
                              "for (int k = 1; k <= p->eps_order; ++k) c *= L;", [pins.test_eps_expansion_d1_against_quad]),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new, checks = MUTATIONS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    src = tmp_path / "oracle_mutant.c"
    src.write_text(text.replace(old, new))
    so = tmp_path / "liboracle_mutant.so"
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-o", str(so), str(src),
                           "-lm", "-lpthread"])
    prev = oracle.use_library(str(so))
    try:
        caught = 0
        for check in checks:
            try:
                check(oracle)
            except AssertionError:
                caught += 1
        assert caught > 0, f"no pin caught the planted mistake {name}"
    finally:
        oracle.use_library(None)
        oracle._lib = prev

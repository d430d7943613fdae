"""qmc_integrate_noalloc: the rule for callers that cannot allocate device
memory (an allocator that is locked, exhausted or owned by a host framework),
with its scratch in a fixed per-device array.  Checked through the C ABI
against qmc_integrate on two calls in a row (the second call finds the first
call's scratch contents and must not depend on them).  Kept in a file of its
own that pytest collects last."""
import numpy as np
import pytest

from paper_1811_11722_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    from paper_1811_11722_gb300 import build, qmc
    build.build_library()
    return qmc


@pytest.mark.parametrize("precision,transform,alpha,tol", [("fp32", "baker", 0, 2e-7), ("fp64", "korobov", 3, 1e-12)])
def test_noalloc_matches_integrate_twice(Q, precision, transform, alpha, tol):
    p = I.config2(n=1000003, m=32)
    p.transform, p.alpha = transform, alpha
    g = I.random_generating_vector(I.SplitMix64(77), p.d, p.n)
    f = Q.integrand_from_problem(p, precision)
    t = Q.transform(transform, alpha)
    ref, ref_ps = Q.qmc_integrate(p.d, p.n, p.m, g, p.shifts, t, f, want_per_shift=True)
    ref = ref.as_dict()
    for _ in range(2):
        res, ps = Q.qmc_integrate_noalloc(p.d, p.n, p.m, g, p.shifts, t, f)
        r = res.as_dict()
        assert r["status"] == 0
        assert np.all(np.abs(ps[:, 0] - ref_ps[:, 0]) <= tol * np.abs(ref_ps[:, 0]))
        assert abs(r["mean"][0] - ref["mean"][0]) <= tol * abs(ref["mean"][0])
        assert abs(r["err"][0] - ref["err"][0]) <= 2 * tol * abs(ref["mean"][0])


def test_noalloc_rejects_oversized_request(Q):
    """More shift slots than the fixed scratch array holds is refused, not
    truncated.  A d = 2 FP64 sector kernel keeps several CTAs per SM, so
    m = 1024 shifts need m x (CTAs of one wave) x 16 B > 4 MiB of slots."""
    rng = I.SplitMix64(5)
    d, n, m = 2, 16777213, 1024
    U = I.random_poly(rng, d, 2, 0)
    F = I.random_poly(rng, d, 0, 3)
    p = I.Problem("big", d, n, m, I.make_shifts(rng, m, d), "baker", kind="sector", U=U, F=F)
    g = I.random_generating_vector(I.SplitMix64(78), d, n)
    with pytest.raises(Q.QmcError) as ei:
        Q.qmc_integrate_noalloc(d, n, m, g, p.shifts, Q.transform("baker"), Q.integrand_from_problem(p, "fp64"))
    assert ei.value.status == Q.QMC_EINVAL
    assert "scratch" in Q.qmc_last_error()

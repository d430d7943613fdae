"""qmc_integrate_noalloc: the rule for callers that cannot allocate device
memory (an allocator that is locked, exhausted or owned by a host framework),
with its scratch in a fixed per-device array.  Checked through the C ABI
against qmc_integrate on two calls in a row.  Before each checked call another
call leaves different contents in the shared array: a different slot layout
(other d, m and n, so a different number of CTAs and shift chunks) and
counted non-finite values, so a call that read slots or counters it did not
write itself would show it.  Kept in a file of its own that pytest collects
last."""
import numpy as np
import pytest

from paper_1811_11722_gb300 import inputs as I

pytestmark = pytest.mark.gpu

SCRATCH_BYTES = 4 << 20  # the fixed per-device array the header documents


@pytest.fixture(scope="module")
def Q():
    from paper_1811_11722_gb300 import build, qmc
    build.build_library()
    return qmc


def _dirty_call(Q, d, n, m, precision, seed):
    """A no-alloc call whose F = 1.5 z_1 vanishes at every lattice point with
    x_1 = 0: with Delta_1 = 0 for every shift, the point j = 0 (and, baker
    being symmetric, no other) gives F = 0, so each shift counts one
    non-finite value."""
    rng = I.SplitMix64(seed)
    U = I.random_poly(rng, d, d, 0)
    F = I.Poly(np.array([1.5]), np.eye(d, dtype=np.uint8)[1:2])
    shifts = I.make_shifts(rng, m, d)
    shifts[:, 1] = 0.0
    p = I.Problem("dirty", d, n, m, shifts, "baker", kind="sector", U=U, F=F, aU=-2, aF=-1)
    g = I.random_generating_vector(I.SplitMix64(seed + 1), d, n)
    res, _ = Q.qmc_integrate_noalloc(d, n, m, g, shifts, Q.transform("baker"), Q.integrand_from_problem(p, precision))
    r = res.as_dict()
    assert r["status"] == Q.QMC_ENONFINITE and r["nonfinite"] == m
    return r


@pytest.mark.parametrize("precision,transform,alpha,tol", [("fp32", "baker", 0, 2e-7), ("fp64", "korobov", 3, 1e-12)])
def test_noalloc_matches_integrate_twice(Q, precision, transform, alpha, tol):
    p = I.config2(n=1000003, m=32)
    p.transform, p.alpha = transform, alpha
    g = I.random_generating_vector(I.SplitMix64(77), p.d, p.n)
    f = Q.integrand_from_problem(p, precision)
    t = Q.transform(transform, alpha)
    ref, ref_ps = Q.qmc_integrate(p.d, p.n, p.m, g, p.shifts, t, f, want_per_shift=True)
    ref = ref.as_dict()
    # before each checked call: a small lattice (few CTAs, 5 shifts), then a
    # d = 2 FP64 rule with 40 shifts on every resident CTA (more slots than the
    # checked call writes)
    for dirty in ((3, 30011, 5, "fp32", 11), (2, 4194301, 40, "fp64", 12)):
        _dirty_call(Q, *dirty)
        res, ps = Q.qmc_integrate_noalloc(p.d, p.n, p.m, g, p.shifts, t, f)
        r = res.as_dict()
        assert r["status"] == 0 and r["nonfinite"] == 0
        assert np.all(np.abs(ps[:, 0] - ref_ps[:, 0]) <= tol * np.abs(ref_ps[:, 0]))
        assert abs(r["mean"][0] - ref["mean"][0]) <= tol * abs(ref["mean"][0])
        assert abs(r["err"][0] - ref["err"][0]) <= 2 * tol * abs(ref["mean"][0])


def test_noalloc_rejects_oversized_request(Q):
    """More shift slots than the fixed scratch array holds is refused, not
    truncated.  The slots take m x (CTAs of one resident wave) x 16 bytes; the
    CTA count is the one the library reports for the same rule through a plan
    (same kernel, same occupancy), and m is chosen so the slots alone exceed
    the array.  Where even m = 1024 fits (one CTA per SM), there is nothing to
    refuse and the test is skipped."""
    rng = I.SplitMix64(5)
    d, n = 2, 16777213
    U = I.random_poly(rng, d, 2, 0)
    F = I.random_poly(rng, d, 0, 3)
    shifts = I.make_shifts(rng, 1024, d)
    g = I.random_generating_vector(I.SplitMix64(78), d, n)
    p = I.Problem("big", d, n, 2, shifts[:2], "baker", kind="sector", U=U, F=F)
    f = Q.integrand_from_problem(p, "fp64")
    ctas = int(Q.Plan(d, n, 16, g, shifts[:16], Q.transform("baker"), f).describe()["ctas"])
    m = SCRATCH_BYTES // (ctas * 16) + 1
    if m > 1024:
        pytest.skip(f"{ctas} CTAs x 1024 shifts of slots fit the {SCRATCH_BYTES}-byte array: nothing to refuse")
    with pytest.raises(Q.QmcError) as ei:
        Q.qmc_integrate_noalloc(d, n, m, g, shifts[:m], Q.transform("baker"), f)
    assert ei.value.status == Q.QMC_EINVAL
    msg = Q.qmc_last_error()
    assert "scratch" in msg and f"on {ctas} CTAs" in msg

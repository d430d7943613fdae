"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.

Tolerances
  * lattice indices: bit-exact.
  * FP64 path: per-shift Q^(k) and Qbar within 1e-12 relative; the error
    estimate within 2e-12 |Qbar| absolute (sigma is a difference of nearly
    equal numbers, so its own relative error is not meaningful).
  * FP32EVAL path: the per-point value carries O(10) float roundings
    (coordinate 2^-24, transform, polynomial, reciprocal), bounded here by
    64 * 2^-24 ~ 4e-6 relative per point; the per-shift sums are compensated
    and promoted to FP64, so Q^(k) differs from the oracle by the average of
    those per-point errors, bounded (worst case, fully correlated) by the same
    4e-6 and typically ~1e-7/sqrt(n).  Tests use 4e-6 for single points and
    2e-7 relative for Q^(k) at n >= 1e4.
"""
import math
import os

import numpy as np
import pytest

from paper_1811_11722_gb300 import inputs as I

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def Q():
    from paper_1811_11722_gb300 import build, qmc
    build.build_library()
    return qmc


@pytest.fixture(scope="module")
def lattices():
    import json
    return {int(k): np.array(v, dtype=np.uint64) for k, v in
            json.load(open(os.path.join(HERE, "golden", "lattices.json")))["g"].items()}


def gvec(lattices, p):
    if p.n in lattices and p.d <= len(lattices[p.n]):
        return lattices[p.n][: p.d]
    return I.random_generating_vector(I.SplitMix64(p.n + p.d), p.d, p.n)


def gpu_run(Q, p, g, precision=None):
    f = Q.integrand_from_problem(p, precision)
    t = Q.transform(p.transform, p.alpha)
    res, ps = Q.qmc_integrate(p.d, p.n, p.m, g, p.shifts, t, f, want_per_shift=True)
    return res.as_dict(), ps


def assert_fp64_parity(gpu, ps, ref):
    q_ref = ref["q"]
    scale = np.max(np.abs(q_ref[:, 0])) + 1e-300
    assert np.all(np.abs(ps[:, 0] - q_ref[:, 0]) <= 1e-12 * np.abs(q_ref[:, 0]) + 1e-15 * scale)
    assert abs(gpu["mean"][0] - ref["mean"][0]) <= 1e-12 * abs(ref["mean"][0]) + 1e-300
    assert abs(gpu["err"][0] - ref["err"][0]) <= 2e-12 * abs(ref["mean"][0]) + 1e-300


# ------------------------------------------------------------ single points --

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("transform,alpha", [("baker", 0), ("korobov", 3), ("none", 0)])
def test_points_sector_d6(Q, oracle_lib, lattices, precision, transform, alpha):
    """Indices bit-exact; coordinates within 2^-52 (FP64) or 2^-23 (FP32) of
    the oracle's; weighted values within 1e-13 / 4e-6 relative, plus, for the
    Korobov weight prod (s_i (1 - s_i))^3 with s_i = min(x_i, 1 - x_i), the
    propagated coordinate error 3 * 2 * dx / s_i per dimension (the weight's
    relative sensitivity near the cube's boundary)."""
    p = I.config2(n=16777213, m=32)
    p.transform, p.alpha = transform, alpha
    g = gvec(lattices, p)
    rng = np.random.default_rng(3)
    js = np.concatenate([[0, 1, 2, p.n - 1, p.n - 2], rng.integers(0, p.n, 200)]).astype(np.uint64)
    ks = np.concatenate([[0, 31, 5, 17, 31], rng.integers(0, p.m, 200)]).astype(np.int32)
    vals, idx, crd = Q.qmc_sample_points(p.d, p.n, p.m, g, p.shifts, Q.transform(transform, alpha),
                                         Q.integrand_from_problem(p, precision), js, ks)
    ctol = 2.0 ** -52 if precision == "fp64" else 2.0 ** -23
    vtol = 1e-13 if precision == "fp64" else 4e-6
    for s in range(len(js)):
        v, oi, ox, _, _ = oracle_lib.point(p, g, int(ks[s]), int(js[s]))
        assert np.array_equal(idx[s], oi)
        dx = np.abs(crd[s] - ox)
        dx = np.minimum(dx, 1.0 - dx)  # coordinates live on the torus
        assert np.all(dx <= ctol), (s, crd[s], ox)
        rel = vtol
        if transform == "korobov":
            sdist = np.minimum(ox, 1.0 - ox)
            rel += float(np.sum(6.0 * ctol / np.maximum(sdist, 1e-300)))
        assert abs(vals[s, 0] - v[0]) <= rel * abs(v[0]) + 1e-300, (s, vals[s, 0], v[0])


def test_points_general_kernel_degree3(Q, oracle_lib):
    """Degree-3 F (the Zbb vertex polynomial of Eq. 11 plus a constant) in d = 6
    goes through the general sparse kernel; values match the oracle."""
    F = I.zbb_vertex_F()
    F = I.Poly(np.concatenate([[4.0], F.coef]), np.vstack([np.zeros((1, 6), np.uint8), F.expo]))
    U = I.random_poly(I.SplitMix64(5), 6, 6, 0)
    rng = I.SplitMix64(6)
    p = I.Problem("zbb", 6, 100003, 4, I.make_shifts(rng, 4, 6), "korobov", alpha=2, kind="sector", U=U, F=F)
    g = I.random_generating_vector(rng, 6, p.n)
    js = np.arange(0, 100003, 997, dtype=np.uint64)
    ks = (np.arange(len(js)) % 4).astype(np.int32)
    vals, idx, _ = Q.qmc_sample_points(p.d, p.n, p.m, g, p.shifts, Q.transform("korobov", 2),
                                       Q.integrand_from_problem(p, "fp64"), js, ks)
    for s in range(len(js)):
        v, oi, _, _, _ = oracle_lib.point(p, g, int(ks[s]), int(js[s]))
        assert np.array_equal(idx[s], oi)
        assert abs(vals[s, 0] - v[0]) <= 1e-12 * abs(v[0]) + 1e-14


# --------------------------------------------------------------- whole rule --

def test_config1_fp64(Q, oracle_lib, lattices):
    """Configuration 1 as specified: d=3 separable exp, Korobov 3, n=10007, m=10."""
    p = I.config1()
    g = gvec(lattices, p)
    gpu, ps = gpu_run(Q, p, g)
    ref = oracle_lib.integrate(p, g)
    assert gpu["status"] == 0
    assert_fp64_parity(gpu, ps, ref)


@pytest.mark.parametrize("transform,alpha", [("baker", 0), ("korobov", 3), ("none", 0)])
def test_sector_d6_fp64_several_tiles(Q, oracle_lib, nthreads, transform, alpha):
    """d=6 sector, n = 100003 (many tiles, ragged tail), m = 20 (two shift chunks)."""
    p = I.config2(n=100003, m=20, precision="fp64")
    p.transform, p.alpha = transform, alpha
    g = I.random_generating_vector(I.SplitMix64(7), 6, p.n)
    gpu, ps = gpu_run(Q, p, g)
    ref = oracle_lib.integrate(p, g, nthreads=nthreads)
    assert_fp64_parity(gpu, ps, ref)


@pytest.mark.parametrize("transform,alpha", [("baker", 0), ("korobov", 3)])
def test_sector_d6_fp32(Q, oracle_lib, nthreads, transform, alpha):
    p = I.config2(n=100003, m=32)
    p.transform, p.alpha = transform, alpha
    g = I.random_generating_vector(I.SplitMix64(8), 6, p.n)
    gpu, ps = gpu_run(Q, p, g, "fp32")
    ref = oracle_lib.integrate(p, g, nthreads=nthreads)
    rel = np.abs(ps[:, 0] - ref["q"][:, 0]) / np.abs(ref["q"][:, 0])
    assert np.all(rel <= 2e-7), (int(np.argmax(rel)), float(rel.max()), ps[:, 0].tolist())
    assert abs(gpu["mean"][0] - ref["mean"][0]) <= 2e-7 * abs(ref["mean"][0])


@pytest.mark.parametrize("d", [1, 2, 3, 4, 5, 7, 8])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_sector_all_dims(Q, oracle_lib, d, precision):
    """Every specialised dimension, with both shift-chunk paths (m = 10)."""
    rng = I.SplitMix64(100 + d)
    U = I.random_poly(rng, d, d, 0)
    F = I.random_poly(rng, d, 0, d * (d + 1) // 2)
    p = I.Problem("sec", d, 20011, 10, I.make_shifts(rng, 10, d), "korobov", alpha=3, kind="sector", U=U, F=F)
    g = I.random_generating_vector(rng, d, p.n)
    gpu, ps = gpu_run(Q, p, g, precision)
    ref = oracle_lib.integrate(p, g)
    if precision == "fp64":
        assert_fp64_parity(gpu, ps, ref)
    else:
        assert np.all(np.abs(ps[:, 0] - ref["q"][:, 0]) <= 4e-7 * np.abs(ref["q"][:, 0]))


@pytest.mark.parametrize("alpha", [1, 2, 4, 5, 6])
def test_korobov_weights_general(Q, oracle_lib, alpha):
    """Korobov weights other than 3 (general kernel for sectors, runtime weight
    for separable integrands)."""
    p = I.config2(n=30011, m=6, precision="fp64")
    p.transform, p.alpha = "korobov", alpha
    g = I.random_generating_vector(I.SplitMix64(alpha), 6, p.n)
    gpu, ps = gpu_run(Q, p, g)
    ref = oracle_lib.integrate(p, g, nthreads=4)
    assert_fp64_parity(gpu, ps, ref)
    c = I.config1(n=30011, m=6)
    c.alpha = alpha
    gpu, ps = gpu_run(Q, c, g[:3])
    assert_fp64_parity(gpu, ps, oracle_lib.integrate(c, g[:3]))


def test_large_d_general_kernel(Q, oracle_lib):
    """d = 12 > 8 sector (general kernel) and d = 16 separable."""
    rng = I.SplitMix64(12)
    U = I.random_poly(rng, 12, 12, 0)
    F = I.random_poly(rng, 12, 0, 20)
    p = I.Problem("d12", 12, 10007, 3, I.make_shifts(rng, 3, 12), "baker", kind="sector", U=U, F=F)
    g = I.random_generating_vector(rng, 12, p.n)
    for prec in ("fp64", "fp32"):
        gpu, ps = gpu_run(Q, p, g, prec)
        ref = oracle_lib.integrate(p, g)
        if prec == "fp64":
            assert_fp64_parity(gpu, ps, ref)
        else:
            assert np.all(np.abs(ps[:, 0] - ref["q"][:, 0]) <= 4e-7 * np.abs(ref["q"][:, 0]))
    c = I.Problem("sep16", 16, 10007, 4, I.make_shifts(rng, 4, 16), "korobov", alpha=6, kind="separable_exp",
                  c=np.linspace(0.1, 0.9, 16), b=np.linspace(0.9, 0.1, 16))
    g16 = I.random_generating_vector(rng, 16, c.n)
    gpu, ps = gpu_run(Q, c, g16)
    assert_fp64_parity(gpu, ps, oracle_lib.integrate(c, g16))


# ------------------------------------------------------------- pinned cases --

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_constant_baker_exact_on_gpu(Q, precision):
    """Sec. 2 / Fig. 3 text: baker on the constant has zero error for any lattice."""
    for d in (6, 9, 10):
        rng = I.SplitMix64(d)
        p = I.Problem("c", d, 100003, 5, I.make_shifts(rng, 5, d), "baker", kind="const")
        g = I.random_generating_vector(rng, d, p.n)
        gpu, ps = gpu_run(Q, p, g, precision)
        assert np.all(ps[:, 0] == 1.0) and gpu["var"][0] == 0.0


def test_dual_lattice_trig_on_gpu(Q):
    """Eq. (2) on cos(2 pi h.x): cos(2 pi h.Delta_k) on the dual lattice, else 0."""
    n, g = 101, np.array([1, 39, 17], dtype=np.uint64)
    sh = I.make_shifts(I.SplitMix64(9), 4, 3)
    for h in ([-39, 1, 0], [17, 0, -1], [1, 1, 0], [3, -2, 5]):
        h = np.array(h, dtype=np.int32)
        p = I.Problem("trig", 3, n, 4, sh, "none", kind="trig", h=h)
        gpu, ps = gpu_run(Q, p, g)
        dual = int(np.dot(h.astype(np.int64), g.astype(np.int64))) % n == 0
        want = np.array([math.cos(2 * math.pi * float(np.dot(h, sh[k]))) if dual else 0.0 for k in range(4)])
        assert np.all(np.abs(ps[:, 0] - want) < 1e-13)


# ---------------------------------------------------------------- edge cases --

@pytest.mark.parametrize("n,d,m", [(2, 1, 2), (3, 2, 2), (257, 3, 33), (65537, 2, 40), (1021, 8, 64)])
def test_edge_sizes(Q, oracle_lib, n, d, m):
    """Smallest lattices, m = 2, m above one launch chunk, ragged tails."""
    rng = I.SplitMix64(n + d + m)
    U = I.random_poly(rng, d, d, 0)
    F = I.random_poly(rng, d, 0, max(1, d))
    p = I.Problem("edge", d, n, m, I.make_shifts(rng, m, d), "baker", kind="sector", U=U, F=F)
    g = np.array([1] + [rng.randint(1, n - 1) for _ in range(d - 1)], dtype=np.uint64)
    gpu, ps = gpu_run(Q, p, g, "fp64")
    assert_fp64_parity(gpu, ps, oracle_lib.integrate(p, g))


@pytest.mark.slow
def test_largest_n(Q, oracle_lib, nthreads):
    """n = 2^31 - 1, the largest lattice the library takes, at d = 2. The
    index products j g reach 2^62 and the fixed-point reciprocal of n is at
    its precision limit.
    * Points at both ends of the index range: indices bit-exact, FP64
      values within 1e-12.
    * The first shift's Q^(1) over all 2.1e9 points against the oracle: FP64
      within 1e-12, FP32 within 2e-7."""
    n, d = 2147483647, 2
    rng = I.SplitMix64(2024)
    U = I.random_poly(rng, d, 2, 0)
    F = I.random_poly(rng, d, 0, 2)
    sh = I.make_shifts(rng, 2, d)
    p = I.Problem("largest_n", d, n, 2, sh, "baker", kind="sector", U=U, F=F)
    g = np.array([1, 1432590847], dtype=np.uint64)
    t = Q.transform("baker")
    js = np.array([0, 1, 2, 1 << 30, (1 << 31) - 3, n - 2, n - 1], dtype=np.uint64)
    ks = np.array([0, 1, 0, 1, 0, 1, 0], dtype=np.int32)
    vals, idx, _ = Q.qmc_sample_points(d, n, 2, g, sh, t, Q.integrand_from_problem(p, "fp64"), js, ks,
                                       want_coord=False)
    for s in range(len(js)):
        v, oi, _, _, _ = oracle_lib.point(p, g, int(ks[s]), int(js[s]))
        assert np.array_equal(idx[s], oi), s
        assert abs(vals[s][0] - v[0]) <= 1e-12 * abs(v[0]), s
    _, ps64 = gpu_run(Q, p, g, "fp64")
    _, ps32 = gpu_run(Q, p, g, "fp32")
    sums, nonf, _ = oracle_lib.rule_sums(p, g, 0, n, nthreads=nthreads, shifts=sh[:1])
    assert int(nonf.sum()) == 0
    ref = sums[0, 0] / n
    assert abs(ps64[0, 0] - ref) <= 1e-12 * abs(ref)
    assert abs(ps32[0, 0] - ref) <= 2e-7 * abs(ref)


def test_nonfinite_values_counted(Q, oracle_lib):
    """F without a constant term vanishes at z = 0: 1/F is infinite there.  Both
    sides leave those points out and count them."""
    d, n, m = 2, 1009, 3
    U = I.Poly(np.array([1.0]), np.zeros((1, d), np.uint8))
    F = I.Poly(np.array([1.0, 1.0]), np.array([[1, 0], [0, 1]], np.uint8))
    sh = np.zeros((m, d))
    sh[1] = [0.5, 0.25]
    p = I.Problem("nf", d, n, m, sh, "baker", kind="sector", U=U, F=F, aU=-2, aF=-1)
    g = np.array([1, 17], dtype=np.uint64)
    gpu, ps = gpu_run(Q, p, g, "fp64")
    ref = oracle_lib.integrate(p, g)
    assert int(ref["nonfinite"].sum()) > 0
    assert gpu["nonfinite"] == int(ref["nonfinite"].sum())
    assert gpu["status"] == Q.QMC_ENONFINITE
    assert np.allclose(ps[:, 0], ref["q"][:, 0], rtol=1e-12)


def test_bit_reproducible(Q, lattices):
    p = I.config2(n=1000003, m=32)
    g = I.random_generating_vector(I.SplitMix64(1), 6, p.n)
    a, pa = gpu_run(Q, p, g, "fp32")
    b, pb = gpu_run(Q, p, g, "fp32")
    assert np.array_equal(pa, pb) and a["mean"][0] == b["mean"][0] and a["var"][0] == b["var"][0]


def test_plan_device_output_matches_host(Q):
    torch = pytest.importorskip("torch")
    p = I.config2(n=1000003, m=32)
    g = I.random_generating_vector(I.SplitMix64(2), 6, p.n)
    f = Q.integrand_from_problem(p, "fp32")
    t = Q.transform("baker")
    plan = Q.Plan(p.d, p.n, p.m, g, p.shifts, t, f)
    host = plan.execute().as_dict()
    out = torch.zeros(Q.RESULT_BYTES, dtype=torch.uint8, device="cuda")
    per = torch.zeros(2 * p.m, dtype=torch.float64, device="cuda")
    plan.execute(out=out, per_shift=per, stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    r = Q.qmc_result.from_buffer_copy(out.cpu().numpy().tobytes()).as_dict()
    assert r["mean"][0] == host["mean"][0] and r["var"][0] == host["var"][0]
    assert plan.launches() == 2
    plan.destroy()


# ------------------------------------------------------------------ full size --

def test_config2_full_size_fp32_vs_oracle(Q, oracle_lib, lattices, nthreads):
    """The benchmark workload (d=6, n=16777213, m=32, baker, FP32EVAL) against the
    oracle over the whole lattice on all host cores."""
    p = I.config2()
    g = gvec(lattices, p)
    gpu, ps = gpu_run(Q, p, g, "fp32")
    ref = oracle_lib.integrate(p, g, nthreads=nthreads)
    rel = np.abs(ps[:, 0] - ref["q"][:, 0]) / np.abs(ref["q"][:, 0])
    assert np.all(rel <= 2e-7), (int(np.argmax(rel)), float(rel.max()), ps[:, 0].tolist())
    assert abs(gpu["mean"][0] - ref["mean"][0]) <= 2e-7 * abs(ref["mean"][0])
    g64, ps64 = gpu_run(Q, p, g, "fp64")
    assert_fp64_parity(g64, ps64, ref)


# -------------------------------------------------------- deformed (complex) --

def _c4(n=100003, m=20, lam=0.1):
    return I.config4(n=n, m=m, lam=lam)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_points_deformed_d5(Q, oracle_lib, precision):
    """Configuration 4 terms: complex values (contour, Jacobian determinant,
    U^-2 F^-1) against the oracle's LU-with-pivoting evaluation."""
    p = _c4(n=4194301)
    g = I.random_generating_vector(I.SplitMix64(41), 5, p.n)
    rng = np.random.default_rng(4)
    js = np.concatenate([[0, 1, p.n - 1], rng.integers(0, p.n, 150)]).astype(np.uint64)
    ks = np.concatenate([[0, 19, 7], rng.integers(0, p.m, 150)]).astype(np.int32)
    vals, idx, _ = Q.qmc_sample_points(p.d, p.n, p.m, g, p.shifts, Q.transform("korobov", 3),
                                       Q.integrand_from_problem(p, precision), js, ks, want_coord=False)
    ctol = 2.0 ** -52 if precision == "fp64" else 2.0 ** -23
    vtol = 1e-12 if precision == "fp64" else 3e-5
    for s in range(len(js)):
        v, oi, ox, _, _ = oracle_lib.point(p, g, int(ks[s]), int(js[s]))
        assert np.array_equal(idx[s], oi)
        sdist = np.minimum(ox, 1.0 - ox)
        rel = vtol + float(np.sum(6.0 * ctol / np.maximum(sdist, 1e-300)))
        mag = abs(complex(v[0], v[1]))
        assert abs(complex(*vals[s]) - complex(v[0], v[1])) <= rel * mag + 1e-300, (s, vals[s], v)


def test_config4_deformed_fp64(Q, oracle_lib, nthreads):
    """Configuration 4 rule (d=5, F with 3 negative coefficients, lambda=0.1,
    Korobov 3, m=20): per-shift complex Q^(k), Qbar, sigma per part, and the
    count of points with Im F(w) > 0, against the oracle."""
    p = _c4()
    g = I.random_generating_vector(I.SplitMix64(42), 5, p.n)
    gpu, ps = gpu_run(Q, p, g)
    ref = oracle_lib.integrate(p, g, nthreads=nthreads)
    scale = np.abs(ref["q"][:, 0] + 1j * ref["q"][:, 1])
    assert np.all(np.abs((ps[:, 0] + 1j * ps[:, 1]) - (ref["q"][:, 0] + 1j * ref["q"][:, 1])) <= 1e-12 * scale)
    mag = abs(complex(*ref["mean"]))
    assert abs(complex(*gpu["mean"]) - complex(*ref["mean"])) <= 1e-12 * mag
    assert np.all(np.abs(gpu["err"] - ref["err"]) <= 2e-12 * mag)
    assert gpu["deform_violations"] == ref["deform_bad"]


def test_config4_deformed_fp32(Q, oracle_lib, nthreads):
    p = _c4()
    g = I.random_generating_vector(I.SplitMix64(43), 5, p.n)
    gpu, ps = gpu_run(Q, p, g, "fp32")
    ref = oracle_lib.integrate(p, g, nthreads=nthreads)
    scale = np.abs(ref["q"][:, 0] + 1j * ref["q"][:, 1])
    assert np.all(np.abs((ps[:, 0] + 1j * ps[:, 1]) - (ref["q"][:, 0] + 1j * ref["q"][:, 1])) <= 2e-6 * scale)


@pytest.mark.slow
def test_config4_full_size(Q, oracle_lib, nthreads):
    """Configuration 4 at its full size (n = 4194301, m = 20), the launch
    configuration the benchmark times, in both precisions.
    * The first two shifts of each against the oracle over every point: FP64
      within 1e-12, FP32 within the small case's 2e-6.
    * The FP32 mean's distance from the FP64 mean within a quarter of the
      Eq. (3) error estimate of each part."""
    import dataclasses
    p = _c4(n=4194301)
    g = I.random_generating_vector(I.SplitMix64(4), 5, p.n)
    g64, ps64 = gpu_run(Q, p, g, "fp64")
    g32, ps32 = gpu_run(Q, p, g, "fp32")
    p2 = dataclasses.replace(p, m=2, shifts=p.shifts[:2].copy())
    ref = oracle_lib.integrate(p2, g, nthreads=nthreads)["q"]
    rc = ref[:, 0] + 1j * ref[:, 1]
    assert np.all(np.abs((ps64[:2, 0] + 1j * ps64[:2, 1]) - rc) <= 1e-12 * np.abs(rc))
    assert np.all(np.abs((ps32[:2, 0] + 1j * ps32[:2, 1]) - rc) <= 2e-6 * np.abs(rc))
    for part in (0, 1):
        assert abs(g32["mean"][part] - g64["mean"][part]) <= 0.25 * g64["err"][part], part


@pytest.mark.slow
def test_fp32_deformed_unbiased_at_full_size(Q):
    """Configuration 4 at full size (n = 4194301, m = 20) in FP32 against FP64
    on the same lattice and shifts.  The FP32 fast variant takes the sector
    kernels' dithered fixed-point coordinates and compensated weight, and
    factors the Jacobian as J = I + B with the identity implicit, carrying
    det J - 1 (rounding each diagonal entry of J near 1 after every small
    elimination update made the integral 2.0e-8 too large).  What remains is
    rounding noise: the per-point FP32 - FP64 difference, measured here on
    2^16 sampled points, has a root mean square s (about 1.7e-6 of |Q|), so a
    per-shift sum over n points scatters by about s / sqrt(n) and the mean
    over m shifts by s / sqrt(n m).  Per shift the difference must stay within
    5 s / sqrt(n) + 1e-10 d, the mean within 5 s / sqrt(n m) + 1e-10 d
    (about 1.4e-9, against the old 2.0e-8), and the sampled points' mean
    difference within 5 s / sqrt(2^16) of zero."""
    p = _c4(n=4194301)
    g = Q.qmc_make_lattice(p.d, p.n, p.gamma)
    _, ps64 = gpu_run(Q, p, g, "fp64")
    _, ps32 = gpu_run(Q, p, g, "fp32")
    c64, c32 = ps64[:, 0] + 1j * ps64[:, 1], ps32[:, 0] + 1j * ps32[:, 1]
    q = abs(c64.mean())
    rng = np.random.default_rng(44)
    S = 1 << 16
    js = rng.integers(0, p.n, S).astype(np.uint64)
    ks = rng.integers(0, p.m, S).astype(np.int32)
    t = Q.transform("korobov", 3)
    v32, _, _ = Q.qmc_sample_points(p.d, p.n, p.m, g, p.shifts, t, Q.integrand_from_problem(p, "fp32"), js, ks,
                                    want_idx=False, want_coord=False)
    v64, _, _ = Q.qmc_sample_points(p.d, p.n, p.m, g, p.shifts, t, Q.integrand_from_problem(p, "fp64"), js, ks,
                                    want_idx=False, want_coord=False)
    dv = (v32[:, 0] - v64[:, 0]) + 1j * (v32[:, 1] - v64[:, 1])
    s = float(np.sqrt(np.mean(np.abs(dv) ** 2)) / q)
    rel = np.abs(c32 - c64) / q
    mean_rel = abs((c32 - c64).mean()) / q
    print(f"C4 FP32 - FP64: per point rms {s:.2e}; per shift max {rel.max():.2e}; mean {mean_rel:.2e}; "
          f"sampled mean {abs(dv.mean()) / q:.2e}")
    assert s < 1e-5
    assert abs(dv.mean()) / q <= 5 * s / np.sqrt(S)
    assert mean_rel <= 5 * s / np.sqrt(p.n * p.m) + 1e-10 * p.d
    assert np.all(rel <= 5 * s / np.sqrt(p.n) + 1e-10 * p.d)


def test_fp32_double_coefficients(Q, oracle_lib, nthreads):
    """FP32EVAL rounds each polynomial coefficient to float (reading R12).
    With coefficients that float32 cannot hold, the FP32 path integrates a
    nearby integrand: every coefficient of U and F is positive, so rounding
    moves U and F by at most 2^-24 relative each and U^-2 F^-1 by at most
    3 x 2^-24 (1.8e-7).  Per shift the FP32 value stays within that bound plus
    the FP32 evaluation bound of the other tests (2e-7) of the oracle with the
    exact coefficients, and within 2e-7 of the oracle with the coefficients
    rounded to float first, which places the rest of the difference in the
    coefficients."""
    import dataclasses
    p = I.config2(n=100003, m=32)
    rng = np.random.default_rng(12)
    U = I.Poly(rng.uniform(0.1, 2.0, p.U.nterms), p.U.expo.copy())
    F = I.Poly(rng.uniform(0.1, 2.0, p.F.nterms), p.F.expo.copy())
    assert np.all(U.coef != U.coef.astype(np.float32)) and np.all(F.coef != F.coef.astype(np.float32))
    p = dataclasses.replace(p, U=U, F=F)
    pf = dataclasses.replace(p, U=I.Poly(U.coef.astype(np.float32).astype(np.float64), U.expo),
                             F=I.Poly(F.coef.astype(np.float32).astype(np.float64), F.expo))
    g = I.random_generating_vector(I.SplitMix64(9), 6, p.n)
    _, ps = gpu_run(Q, p, g, "fp32")
    q_exact = oracle_lib.integrate(p, g, nthreads=nthreads)["q"][:, 0]
    q_round = oracle_lib.integrate(pf, g, nthreads=nthreads)["q"][:, 0]
    coef_bound = 3 * 2.0 ** -24
    assert np.all(np.abs(q_round - q_exact) <= coef_bound * np.abs(q_exact))
    assert np.all(np.abs(ps[:, 0] - q_exact) <= (2e-7 + coef_bound) * np.abs(q_exact))
    assert np.all(np.abs(ps[:, 0] - q_round) <= 2e-7 * np.abs(q_round))


@pytest.mark.parametrize("d", [2, 3, 5])
def test_deformed_packed_matches_one_shift_kernel(Q, oracle_lib, nthreads, monkeypatch, d):
    """The FP32 deformed kernel that evaluates two shifts per instruction
    against the one-shift kernel (QMC_DEFORMED_PACKED=0) and the oracle.
    m = 7 leaves the last shift unpaired.  The two kernels differ only in
    rounding (a packed reciprocal), so their per-shift values agree far
    inside the FP32 bound, and both count the same contour violations."""
    rng = I.SplitMix64(4400 + d)
    U = I.random_poly(rng, d, d, 0)
    F = I.random_poly(rng, d, 0, 2 * d, neg_quad=1)
    p = I.Problem(f"def_d{d}", d, 50021, 7, I.make_shifts(rng, 7, d), "korobov", alpha=3,
                  kind="sector_deformed", U=U, F=F, lam=0.1, precision="fp32")
    g = I.random_generating_vector(rng, d, p.n)
    a, pa = gpu_run(Q, p, g, "fp32")
    monkeypatch.setenv("QMC_DEFORMED_PACKED", "0")
    b, pb = gpu_run(Q, p, g, "fp32")
    ca, cb = pa[:, 0] + 1j * pa[:, 1], pb[:, 0] + 1j * pb[:, 1]
    assert np.all(np.abs(ca - cb) <= 1e-6 * np.abs(cb))
    assert a["deform_violations"] == b["deform_violations"] and a["nonfinite"] == b["nonfinite"]
    ref = oracle_lib.integrate(p, g, nthreads=nthreads)
    rc = ref["q"][:, 0] + 1j * ref["q"][:, 1]
    assert np.all(np.abs(ca - rc) <= 2e-6 * np.abs(rc))


def test_deformed_lambda_zero_equals_real_kernel(Q):
    """With lambda = 0 the contour is the real cube and J = I: the complex
    kernel reproduces the real sector kernel (positive F) to rounding."""
    rng = I.SplitMix64(44)
    U = I.random_poly(rng, 4, 4, 0)
    F = I.random_poly(rng, 4, 0, 6)
    sh = I.make_shifts(rng, 6, 4)
    g = I.random_generating_vector(rng, 4, 50021)
    real = I.Problem("r", 4, 50021, 6, sh, "korobov", alpha=3, kind="sector", U=U, F=F)
    cplx = I.Problem("c", 4, 50021, 6, sh, "korobov", alpha=3, kind="sector_deformed", U=U, F=F, lam=0.0)
    a, pa = gpu_run(Q, real, g, "fp64")
    b, pb = gpu_run(Q, cplx, g, "fp64")
    assert np.allclose(pa[:, 0], pb[:, 0], rtol=1e-13, atol=0) and np.all(pb[:, 1] == 0.0)


# -------------------------------------------------------------------- batch --

def _batch_tuple(Q, p, g, precision=None):
    return (p.d, p.n, p.m, g, p.shifts, Q.transform(p.transform, p.alpha), Q.integrand_from_problem(p, precision))


def test_batch_matches_oracle_per_problem(Q, oracle_lib, nthreads):
    """A mixed batch (FP32 sectors of d = 2..8 from the batched-sector
    generator at reduced n, an FP64 separable problem, a deformed FP64
    problem): every problem's per-shift values match the oracle."""
    sect = I.config3(count=10)
    probs = []
    for s, p in enumerate(sect):
        p.n = I.prev_prime(20000 + 3000 * s)
        probs.append(p)
    probs.append(I.config1())
    probs.append(_c4(n=20011, m=8))
    gs = [I.random_generating_vector(I.SplitMix64(500 + i), p.d, p.n) for i, p in enumerate(probs)]
    tuples = [_batch_tuple(Q, p, g) for p, g in zip(probs, gs)]
    res, ps = Q.qmc_integrate_batch(tuples, want_per_shift=True)
    off = 0
    for p, g, r in zip(probs, gs, res):
        ref = oracle_lib.integrate(p, g, nthreads=nthreads)
        q = ps[2 * off: 2 * (off + p.m)].reshape(p.m, 2)
        off += p.m
        refc = ref["q"][:, 0] + 1j * ref["q"][:, 1]
        tol = 4e-7 if p.precision == "fp32" else 1e-12
        assert np.all(np.abs((q[:, 0] + 1j * q[:, 1]) - refc) <= tol * np.abs(refc)), p.name
        assert r.status == 0


def test_batch_plan_graph_replay_and_tune(Q):
    """The batch plan builds its CUDA graph once; replays give identical
    results, tuning keeps results within FP32 rounding, and the launch count
    is one per (problem, shift chunk) plus the final pass."""
    sect = I.config3(count=24)
    for s, p in enumerate(sect):
        p.n = I.prev_prime(50000 + 7000 * s)
    gs = [I.random_generating_vector(I.SplitMix64(700 + i), p.d, p.n) for i, p in enumerate(sect)]
    tuples = [_batch_tuple(Q, p, g) for p, g in zip(sect, gs)]
    bp = Q.BatchPlan(tuples)
    a = [r.as_dict() for r in bp.execute()]
    b = [r.as_dict() for r in bp.execute()]
    for x, y in zip(a, b):
        assert x["mean"][0] == y["mean"][0] and x["var"][0] == y["var"][0]
    assert bp.launches() == len(sect) + 1
    w = bp.tune()
    assert (1 << 18) <= w <= (1 << 24)
    c = [r.as_dict() for r in bp.execute()]
    for x, y in zip(a, c):
        assert abs(x["mean"][0] - y["mean"][0]) <= 1e-7 * abs(x["mean"][0])
    bp.destroy()


def _walk_targets(Q, res, tol, criterion):
    """Each problem's error target: its share of the sum's tolerance, or its own."""
    if criterion == Q.WALK_SUM:
        tot = math.hypot(sum(r.mean[0] for r in res), sum(r.mean[1] for r in res))
        return [tol * tot / math.sqrt(len(res))] * len(res)
    return [tol * math.hypot(r.mean[0], r.mean[1]) for r in res]


def _jump_short(q, excess):
    """QMC_WALK_JUMP's test: a size ratio q still short of the excess,
    q^6 < excess (the product taken in the library's order)."""
    p = 1.0
    for _ in range(6):
        p *= q
    return p < excess


def _excess(r, target):
    return math.hypot(r.err[0], r.err[1]) / target if target > 0 else 1.0


def _python_batch_walk(Q, tuples, ladder_n, ladder_g, tol, criterion, jump=False):
    """The walk of qmc_integrate_batch_to_tolerance written with one
    qmc_integrate_batch call per pass (same lattices, same decisions)."""
    S, L = len(tuples), len(ladder_n)
    nxt = [int(np.searchsorted(ladder_n, t[1], side="right")) for t in tuples]
    at = [-1] * S
    cur = list(tuples)
    res = [None] * S
    act, passes, reached = list(range(S)), 0, False
    while True:
        if passes:
            for i in act:
                l = nxt[i]
                d = cur[i][0]
                cur[i] = (d, int(ladder_n[l]), cur[i][2], ladder_g[l, :d].copy()) + tuple(cur[i][4:])
                at[i], nxt[i] = l, l + 1
        rs, _ = Q.qmc_integrate_batch([cur[i] for i in act])
        for i, r in zip(act, rs):
            res[i] = r
        passes += 1
        mag = [math.hypot(r.mean[0], r.mean[1]) for r in res]
        err = [math.hypot(r.err[0], r.err[1]) for r in res]
        if criterion == Q.WALK_SUM:
            tot = math.hypot(sum(r.mean[0] for r in res), sum(r.mean[1] for r in res))
            if tot > 0 and math.sqrt(sum(e * e for e in err)) <= tol * tot:
                reached = True
                break
            share = tol * tot / math.sqrt(S)
            act = [i for i in range(S) if err[i] > share and nxt[i] < L]
        else:
            ok = [mag[i] > 0 and err[i] <= tol * mag[i] for i in range(S)]
            if all(ok):
                reached = True
                break
            act = [i for i in range(S) if not ok[i] and nxt[i] < L]
        if not act:
            break
        if jump:
            tgt = _walk_targets(Q, res, tol, criterion)
            for i in act:
                ex = _excess(res[i], tgt[i])
                l = nxt[i]
                while l + 1 < L and _jump_short(float(ladder_n[l]) / float(cur[i][1]), ex):
                    l += 1
                nxt[i] = l
    return res, at, passes, reached


@pytest.mark.parametrize("criterion,tol,jump", [("sum", 3e-8, False), ("each", 2e-7, False), ("sum", 1e-15, False),
                                                ("sum", 3e-8, True), ("each", 2e-7, True)])
def test_batch_walk_matches_per_pass_batches(Q, criterion, tol, jump):
    """The batched ladder walk (plans built once, moved to each new lattice)
    against the same walk made of one qmc_integrate_batch per pass: the same
    passes and final lattices, and bit-identical results.  The batch mixes
    FP32 sectors (baker, Korobov 3), an FP64 separable problem and a deformed
    FP64 problem (whose launch shape ignores the CTA cap); the third case's
    tolerance cannot be met, so the ladder runs out.  With QMC_WALK_JUMP a
    problem may skip ladder lattices; the replica takes the same jumps."""
    crit = Q.WALK_SUM if criterion == "sum" else Q.WALK_EACH
    sect = I.config3(count=12, transform="korobov", alpha=3)
    probs = []
    for s, p in enumerate(sect):
        p.n = I.prev_prime(20000 + 9000 * s)
        if s % 3 == 0:
            p.transform, p.alpha = "baker", 0
        probs.append(p)
    probs.append(I.config1())
    probs.append(_c4(n=20011, m=8))
    gs = [I.random_generating_vector(I.SplitMix64(800 + i), p.d, p.n) for i, p in enumerate(probs)]
    tuples = [_batch_tuple(Q, p, g) for p, g in zip(probs, gs)]
    ladder_n = np.array([I.prev_prime(v) for v in (40000, 90000, 200000, 450000, 1000000, 2200000)], np.uint64)
    ladder_g = np.stack([I.random_generating_vector(I.SplitMix64(900 + l), 8, int(n))
                         for l, n in enumerate(ladder_n)]).astype(np.uint64)
    res, lv, passes, reached = Q.qmc_integrate_batch_to_tolerance(tuples, ladder_n, ladder_g, tol,
                                                                  crit | (Q.WALK_JUMP if jump else 0))
    ref, at, ref_passes, ref_reached = _python_batch_walk(Q, tuples, ladder_n, ladder_g, tol, crit, jump)
    assert passes == ref_passes and reached == ref_reached
    assert list(lv) == at
    assert passes >= 2  # at least one move to a ladder lattice
    for r, q in zip(res, ref):
        assert r.mean[0] == q.mean[0] and r.mean[1] == q.mean[1]
        assert r.err[0] == q.err[0] and r.err[1] == q.err[1]
        assert r.nonfinite == q.nonfinite
    if tol < 1e-12:
        assert not reached and passes >= 3


def test_batch_walk_persistent_passes(Q):
    """The walk with persistent passes (one launch of the run-time-lattice
    kernel per pass) against the walk with one kernel per sector: the same
    passes and final lattices, results within the grouping of the sums; and
    every problem's final result equal, bit for bit, to the persistent batch
    plan at its final lattice (the same work items of 2^15 points)."""
    sect = I.config3(count=12, transform="korobov", alpha=3)
    for s, p in enumerate(sect):
        p.n = I.prev_prime(20000 + 9000 * s)
        if s % 3 == 0:
            p.transform, p.alpha = "baker", 0
    gs = [I.random_generating_vector(I.SplitMix64(800 + i), p.d, p.n) for i, p in enumerate(sect)]
    tuples = [_batch_tuple(Q, p, g) for p, g in zip(sect, gs)]
    ladder_n = np.array([I.prev_prime(v) for v in (40000, 90000, 200000, 450000, 1000000, 2200000)], np.uint64)
    ladder_g = np.stack([I.random_generating_vector(I.SplitMix64(900 + l), 8, int(n))
                         for l, n in enumerate(ladder_n)]).astype(np.uint64)
    tol = 3e-8
    res, lv, passes, reached = Q.qmc_integrate_batch_to_tolerance(tuples, ladder_n, ladder_g, tol,
                                                                  Q.WALK_SUM | Q.WALK_PERSISTENT)
    ref, lv_ref, passes_ref, reached_ref = Q.qmc_integrate_batch_to_tolerance(tuples, ladder_n, ladder_g, tol)
    assert passes == passes_ref and reached == reached_ref and list(lv) == list(lv_ref)
    assert passes >= 2
    # the same FP32 values, summed in other groups (items of 2^15 points
    # against CTA tiles): baker's FP32 runs of 8 values round differently, a
    # few 1e-10 of the mean at these n (measured up to 1.5e-10)
    for r, q in zip(res, ref):
        assert abs(r.mean[0] - q.mean[0]) <= 2e-9 * abs(q.mean[0]) and r.nonfinite == q.nonfinite
    final = [(t[0], int(ladder_n[l]) if l >= 0 else t[1], t[2], ladder_g[l, :t[0]].copy() if l >= 0 else t[3])
             + tuple(t[4:]) for t, l in zip(tuples, lv)]
    pp = Q.BatchPlan(final, persistent=True, chunk=1 << 15)
    want = pp.execute()
    pp.destroy()
    for r, q in zip(res, want):
        assert r.mean[0] == q.mean[0] and r.err[0] == q.err[0] and r.nonfinite == q.nonfinite


def _embedded_g(seed, d=8):
    """An odd generating vector for embedded base-2 lattices (g_1 = 1)."""
    rng = I.SplitMix64(seed)
    return np.array([1] + [2 * rng.randint(0, (1 << 29) - 1) + 1 for _ in range(d - 1)], dtype=np.uint64)


def _extensible_problems(Q, seed=0):
    """FP32 sectors (baker, Korobov 3) of d = 2..8, an FP64 separable problem
    and a deformed FP64 problem, each starting at its own power of two."""
    sect = I.config3(count=10, transform="korobov", alpha=3)
    probs = []
    for s, p in enumerate(sect):
        p.n = 1 << (12 + s % 4)
        if s % 3 == 0:
            p.transform, p.alpha = "baker", 0
        probs.append(p)
    c1 = I.config1()
    c1.n = 1 << 13
    probs.append(c1)
    probs.append(_c4(n=1 << 14, m=8))
    return probs


def _shifted_tuple(t, g, n, new_points):
    """Problem tuple t at size n on g mod n; with new_points, the points of
    size 2n that are not in size n (shifts moved by (g mod 2n) / (2n))."""
    d = t[0]
    sh = np.asarray(t[4], dtype=np.float64)
    if new_points:
        v = sh + (g[:d] % np.uint64(2 * n)).astype(np.float64) / float(2 * n)
        sh = np.where(v >= 1.0, v - 1.0, v)
    return (d, n, t[2], g[:d] % np.uint64(n), np.ascontiguousarray(sh)) + tuple(t[5:])


def _python_batch_extensible(Q, tuples, g, levels, tol, criterion, jump=False):
    """The walk of qmc_integrate_batch_extensible written with one
    qmc_integrate_batch call per pass (same points, same decisions), the
    per-shift values averaged and combined on the host.  A jump of k > 1
    doublings evaluates the whole rule of the new size."""
    S = len(tuples)
    size = [t[1] for t in tuples]
    maxd = [min(levels, 30 - int(t[1]).bit_length() + 1) for t in tuples]
    dbl = [0] * S
    step = [1] * S
    q = [None] * S
    res = [None] * S
    act, passes, reached = list(range(S)), 0, False
    while True:
        batch = []
        for i in act:
            if passes > 0 and step[i] > 1:
                batch.append(_shifted_tuple(tuples[i], g, size[i] << step[i], False))
            else:
                batch.append(_shifted_tuple(tuples[i], g, size[i], passes > 0))
        rs, ps = Q.qmc_integrate_batch(batch, want_per_shift=True)
        off = 0
        for i, r in zip(act, rs):
            m = tuples[i][2]
            qn = ps[2 * off: 2 * (off + m)].reshape(m, 2)
            off += m
            if passes == 0:
                q[i] = qn.copy()
            elif step[i] > 1:
                q[i] = qn.copy()
                size[i] <<= step[i]
                dbl[i] += step[i]
            else:
                q[i] = 0.5 * (q[i] + qn)
                size[i] *= 2
                dbl[i] += 1
            res[i] = Q.qmc_combine_shifts(q[i])
        passes += 1
        mag = [math.hypot(r.mean[0], r.mean[1]) for r in res]
        err = [math.hypot(r.err[0], r.err[1]) for r in res]
        if criterion == Q.WALK_SUM:
            tot = math.hypot(sum(r.mean[0] for r in res), sum(r.mean[1] for r in res))
            if tot > 0 and math.sqrt(sum(e * e for e in err)) <= tol * tot:
                reached = True
                break
            share = tol * tot / math.sqrt(S)
            act = [i for i in range(S) if err[i] > share and dbl[i] < maxd[i]]
        else:
            ok = [mag[i] > 0 and err[i] <= tol * mag[i] for i in range(S)]
            if all(ok):
                reached = True
                break
            act = [i for i in range(S) if not ok[i] and dbl[i] < maxd[i]]
        if not act:
            break
        if jump:
            tgt = _walk_targets(Q, res, tol, criterion)
            for i in act:
                ex = _excess(res[i], tgt[i])
                k = 1
                while k < maxd[i] - dbl[i] and _jump_short(float(1 << k), ex):
                    k += 1
                step[i] = k
    return res, dbl, passes, reached


@pytest.mark.parametrize("criterion,tol,levels,jump", [("sum", 3e-8, 8, False), ("each", 2e-7, 8, False),
                                                       ("sum", 1e-15, 3, False), ("sum", 3e-8, 8, True),
                                                       ("each", 2e-7, 8, True), ("sum", 1e-15, 5, True)])
def test_batch_extensible_matches_per_pass_batches(Q, criterion, tol, levels, jump):
    """The batched embedded-lattice walk (plans built once, moved to each
    size and shifted to its new points) against the same walk made of one
    qmc_integrate_batch per pass: the same passes and doublings, and
    bit-identical results.  The third case's tolerance cannot be met, so
    every problem takes its three doublings.  With QMC_WALK_JUMP a problem
    may take several doublings in one pass (the whole rule of its new size);
    in the last case every problem reaches its limit in fewer passes."""
    crit = (Q.WALK_SUM if criterion == "sum" else Q.WALK_EACH) | (Q.WALK_JUMP if jump else 0)
    base_crit = Q.WALK_SUM if criterion == "sum" else Q.WALK_EACH
    probs = _extensible_problems(Q)
    g = _embedded_g(31)
    tuples = [_batch_tuple(Q, p, g[:p.d] % np.uint64(p.n)) for p in probs]
    res, lv, passes, reached = Q.qmc_integrate_batch_extensible(tuples, levels, g, tol, crit)
    ref, dbl, ref_passes, ref_reached = _python_batch_extensible(Q, tuples, g, levels, tol, base_crit, jump)
    assert passes == ref_passes and reached == ref_reached
    assert list(lv) == dbl
    assert passes >= 2
    for r, q in zip(res, ref):
        assert r.mean[0] == q.mean[0] and r.mean[1] == q.mean[1]
        assert r.err[0] == q.err[0] and r.err[1] == q.err[1]
    if tol < 1e-12:
        assert not reached and all(v == levels for v in lv)
        # one doubling per pass, or jumps of up to 64^k in the error: fewer passes
        assert passes == levels + 1 if not jump else passes < levels + 1


def test_batch_extensible_is_the_rule_of_its_size(Q, oracle_lib, nthreads):
    """Each result of the batched embedded-lattice walk is the rule of its
    final size 2^k on g mod 2^k: per problem against qmc_integrate at that
    size (FP32 within its rounding, FP64 within 1e-12), and the FP64
    separable problem against the oracle."""
    probs = _extensible_problems(Q)
    g = _embedded_g(32)
    tuples = [_batch_tuple(Q, p, g[:p.d] % np.uint64(p.n)) for p in probs]
    res, lv, passes, reached = Q.qmc_integrate_batch_extensible(tuples, 3, g, 1e-15, Q.WALK_SUM)
    assert not reached and all(v == 3 for v in lv)
    for p, t, r, l in zip(probs, tuples, res, lv):
        n = p.n << int(l)
        direct, _ = Q.qmc_integrate(p.d, n, p.m, g[:p.d] % np.uint64(n), p.shifts, t[5], t[6])
        tol = 2e-7 if p.precision == "fp32" else 1e-12
        mag = math.hypot(direct.mean[0], direct.mean[1])
        assert math.hypot(r.mean[0] - direct.mean[0], r.mean[1] - direct.mean[1]) <= tol * mag, p.name
        assert math.hypot(r.err[0] - direct.err[0], r.err[1] - direct.err[1]) <= 10 * tol * mag, p.name
        assert r.nonfinite == direct.nonfinite
    p, r = probs[-2], res[-2]
    p.n = p.n << int(lv[-2])
    ref = oracle_lib.integrate(p, g[:p.d] % np.uint64(p.n), nthreads=nthreads)
    assert abs(r.mean[0] - ref["mean"][0]) <= 1e-12 * abs(ref["mean"][0])


def test_batch_walk_without_ladder_is_one_batch(Q):
    """A walk with no ladder lattices evaluates every problem once, on its own
    lattice, exactly as qmc_integrate_batch does, and reports whether the sum
    met the tolerance."""
    sect = I.config3(count=6)
    for s, p in enumerate(sect):
        p.n = I.prev_prime(30000 + 5000 * s)
    gs = [I.random_generating_vector(I.SplitMix64(40 + i), p.d, p.n) for i, p in enumerate(sect)]
    tuples = [_batch_tuple(Q, p, g) for p, g in zip(sect, gs)]
    ref, _ = Q.qmc_integrate_batch(tuples)
    for tol, want in ((1e-15, False), (1.0, True)):
        res, lv, passes, reached = Q.qmc_integrate_batch_to_tolerance(tuples, [], np.zeros((0, 8), np.uint64), tol)
        assert passes == 1 and reached == want and list(lv) == [-1] * len(sect)
        for r, q in zip(res, ref):
            assert r.mean[0] == q.mean[0] and r.err[0] == q.err[0]


def test_persistent_batch_matches_oracle_and_graph(Q, oracle_lib, nthreads):
    """One persistent launch over a mixed batch of FP32 sectors (d = 1..8;
    baker, none and Korobov 3; m = 5, 16 and 21, so shift chunks of 8 with
    padded rows; a non-positive F, so the non-finite check is on): every
    problem's per-shift values match the oracle, and the graph batch on the
    same problems within the grouping of the compensated sums.  Chunks of
    1024 points leave ragged last items."""
    sect = I.config3(count=9)
    trs = [("baker", 0), ("none", 0), ("korobov", 3)]
    ms = [5, 16, 21]
    probs = []
    for s, p in enumerate(sect):
        p.n = I.prev_prime(20000 + 3000 * s)
        p.transform, p.alpha = trs[s % 3]
        p = I.with_shifts(p, ms[s % 3], 1200 + s)
        probs.append(p)
    d1 = I.Problem("d1", 1, 10007, 4, I.make_shifts(I.SplitMix64(5), 4, 1), "baker", kind="sector",
                   U=I.random_poly(I.SplitMix64(6), 1, 1, 0), F=I.random_poly(I.SplitMix64(7), 1, 0, 1),
                   precision="fp32", gamma=I.product_weights(1))
    probs.append(d1)
    neg = I.config3(count=3, seed=I.SEED_BASE + 78)[2]
    neg.n = I.prev_prime(30000)
    neg.F.coef[-1] = -0.05  # F may vanish inside the cube: CHECK path
    probs.append(neg)
    gs = [I.random_generating_vector(I.SplitMix64(800 + i), p.d, p.n) for i, p in enumerate(probs)]
    tuples = [_batch_tuple(Q, p, g, "fp32") for p, g in zip(probs, gs)]
    total_m = sum(p.m for p in probs)
    pp = Q.BatchPlan(tuples, persistent=True, chunk=1024)
    assert pp.launches() == 2
    ps_p = np.zeros(2 * total_m)
    res_p = pp.execute(per_shift=ps_p)
    ps_p2 = np.zeros(2 * total_m)
    pp.execute(per_shift=ps_p2)
    assert np.array_equal(ps_p, ps_p2)  # replays are deterministic
    pp.destroy()
    res_g, ps_g = Q.qmc_integrate_batch(tuples, want_per_shift=True)
    off = 0
    for p, g, r, rg in zip(probs, gs, res_p, res_g):
        q = ps_p[2 * off: 2 * (off + p.m)].reshape(p.m, 2)
        qg = ps_g[2 * off: 2 * (off + p.m)].reshape(p.m, 2)
        off += p.m
        assert r.status == rg.status, p.name
        assert r.nonfinite == rg.nonfinite, p.name
        assert np.all(np.abs(q[:, 0] - qg[:, 0]) <= 1e-8 * np.abs(qg[:, 0])), p.name
        ref = oracle_lib.integrate(p, g, nthreads=nthreads)
        assert np.all(np.abs(q[:, 0] - ref["q"][:, 0]) <= 4e-7 * np.abs(ref["q"][:, 0])), p.name


def test_persistent_specialised_matches_generic(Q, monkeypatch):
    """The persistent batch's run-time specialised kernel (per descriptor:
    straight-line code with the lattice, shifts and nonzero coefficients as
    constants, linked into one module) against the generic persistent kernel
    (QMC_PERSIST_JIT=0: dense coefficients staged in shared memory) on a mixed
    batch: d = 1..8; baker, none and Korobov 3; m = 5, 16 and 21 (descriptors
    of 16 shifts and a ragged 5, padded to an even row count); a non-positive
    F (the non-finite check).  Every value is computed by the same arithmetic
    in the same order and every work item writes its fixed slots, so the
    per-shift results must be bit-identical, and so must the non-finite
    counts."""
    sect = I.config3(count=9)
    trs = [("baker", 0), ("none", 0), ("korobov", 3)]
    ms = [5, 16, 21]
    probs = []
    for s, p in enumerate(sect):
        p.n = I.prev_prime(20000 + 3000 * s)
        p.transform, p.alpha = trs[s % 3]
        probs.append(I.with_shifts(p, ms[s % 3], 1300 + s))
    d1 = I.Problem("d1", 1, 10007, 4, I.make_shifts(I.SplitMix64(15), 4, 1), "korobov", alpha=3, kind="sector",
                   U=I.random_poly(I.SplitMix64(16), 1, 1, 0), F=I.random_poly(I.SplitMix64(17), 1, 0, 1),
                   precision="fp32", gamma=I.product_weights(1))
    probs.append(d1)
    neg = I.config3(count=3, seed=I.SEED_BASE + 79)[2]
    neg.n = I.prev_prime(30000)
    neg.F.coef[-1] = -0.05
    probs.append(neg)
    gs = [I.random_generating_vector(I.SplitMix64(900 + i), p.d, p.n) for i, p in enumerate(probs)]
    tuples = [_batch_tuple(Q, p, g, "fp32") for p, g in zip(probs, gs)]
    total_m = sum(p.m for p in probs)
    spec = Q.BatchPlan(tuples, persistent=True, chunk=2048)
    desc = spec.describe()
    assert desc["specialised"] == "1" and desc["shifts_per_descriptor"] == "16", desc
    assert int(desc["descriptors"]) == sum((p.m + 15) // 16 for p in probs)
    ps_s = np.zeros(2 * total_m)
    res_s = [r.as_dict() for r in spec.execute(per_shift=ps_s)]
    spec.destroy()
    monkeypatch.setenv("QMC_PERSIST_JIT", "0")
    gen = Q.BatchPlan(tuples, persistent=True, chunk=2048)
    assert gen.describe()["specialised"] == "0"
    ps_g = np.zeros(2 * total_m)
    res_g = [r.as_dict() for r in gen.execute(per_shift=ps_g)]
    gen.destroy()
    assert np.array_equal(ps_s, ps_g)
    for a, b in zip(res_s, res_g):
        assert a["mean"][0] == b["mean"][0] and a["nonfinite"] == b["nonfinite"] and a["status"] == b["status"]
    assert res_s[-1]["nonfinite"] > 0 or res_s[-1]["status"] == 0


def test_persistent_batch_tune(Q):
    """The tuner sweeps the work-item size of a persistent plan and keeps
    results within FP32 rounding."""
    sect = I.config3(count=12)
    for s, p in enumerate(sect):
        p.n = I.prev_prime(60000 + 9000 * s)
    gs = [I.random_generating_vector(I.SplitMix64(950 + i), p.d, p.n) for i, p in enumerate(sect)]
    tuples = [_batch_tuple(Q, p, g) for p, g in zip(sect, gs)]
    pp = Q.BatchPlan(tuples, persistent=True)
    a = [r.as_dict() for r in pp.execute()]
    w = pp.tune()
    assert (1 << 14) <= w <= (1 << 18)
    b = [r.as_dict() for r in pp.execute()]
    for x, y in zip(a, b):
        assert abs(x["mean"][0] - y["mean"][0]) <= 1e-7 * abs(x["mean"][0])
    pp.destroy()


def test_config3_full_batch_sampled(Q, oracle_lib, nthreads):
    """The full batched-sector configuration (256 sectors, ~9.3e9 evaluations):
    every status OK, and the six smallest sectors checked against the oracle."""
    sect = I.config3()
    gs = [I.random_generating_vector(I.SplitMix64(900 + i), p.d, p.n) for i, p in enumerate(sect)]
    tuples = [_batch_tuple(Q, p, g) for p, g in zip(sect, gs)]
    res, ps = Q.qmc_integrate_batch(tuples, want_per_shift=True)
    assert all(r.status == 0 for r in res)
    # the same batch as one persistent launch: every sector's per-shift values
    # agree with the graph's within the grouping of the compensated sums
    pp = Q.BatchPlan(tuples, persistent=True)
    ps_p = np.zeros_like(ps)
    assert all(r.status == 0 for r in pp.execute(per_shift=ps_p))
    assert np.all(np.abs(ps_p[0::2] - ps[0::2]) <= 1e-8 * np.abs(ps[0::2]))
    # tuned (item size, and one or two CTAs per SM for the specialised kernel):
    # the same values up to the grouping of the sums into items
    pp.tune()
    ps_t = np.zeros_like(ps)
    assert all(r.status == 0 for r in pp.execute(per_shift=ps_t))
    pp.destroy()
    assert np.all(np.abs(ps_t[0::2] - ps[0::2]) <= 1e-8 * np.abs(ps[0::2]))
    offs = np.cumsum([0] + [p.m for p in sect])
    for i in sorted(range(len(sect)), key=lambda i: sect[i].n)[:6]:
        ref = oracle_lib.integrate(sect[i], gs[i], nthreads=nthreads)
        q = ps[2 * offs[i]: 2 * offs[i + 1]].reshape(sect[i].m, 2)
        assert np.all(np.abs(q[:, 0] - ref["q"][:, 0]) <= 4e-7 * np.abs(ref["q"][:, 0]))


def test_plan_tune_keeps_results(Q):
    p = I.config2(n=1000003, m=32)
    g = I.random_generating_vector(I.SplitMix64(3), 6, p.n)
    plan = Q.Plan(p.d, p.n, p.m, g, p.shifts, Q.transform("baker"), Q.integrand_from_problem(p, "fp32"))
    a = plan.execute().as_dict()
    mc = plan.tune()
    assert mc in (8, 16, 32)
    b = plan.execute().as_dict()
    assert abs(a["mean"][0] - b["mean"][0]) <= 1e-7 * abs(a["mean"][0])
    plan.destroy()


# ---------------------------------------------------------- control variate --

def _cv_cfg(Q, steps=300, freq=1, seed=7):
    import ctypes
    cfg = Q.qmc_cv_config()
    cfg.R, cfg.K, cfg.freq_step, cfg.steps, cfg.lr, cfg.seed = 16, 32, freq, steps, 1e-2, seed
    return cfg


@pytest.mark.parametrize("d,P", [(8, 3000), (3, 1000), (1, 77)])
def test_cv_gradient_matches_oracle(Q, oracle_lib, d, P):
    """Training kernels (BF16 tensor-core contractions, FP32 accumulation)
    against the oracle's chain rule on the same BF16-rounded operands with FP64
    sums: what differs is FP32 accumulation and, rarely, the BF16 rounding of a
    gradient factor computed in FP32 instead of FP64.  Pilot sizes that are
    not multiples of the 64-point tile check the padding.  Against the all-FP64
    fit the difference stays within BF16's resolution."""
    rng = np.random.default_rng(11)
    a = (rng.normal(size=16 * d * 32) * 0.05).astype(np.float32)
    a[[(r * d + i) * 32 for r in range(16) for i in range(d)]] = 0.8
    x = rng.random((P, d))
    h = rng.random(P)
    loss, grad = Q.qmc_cv_loss_grad(d, _cv_cfg(Q), x, h, a)
    lref, gref = oracle_lib.cv_loss_grad_bf16(d, 16, 32, 1, x, h, a)
    assert abs(loss - lref) <= 1e-5 * lref
    assert np.max(np.abs(grad - gref)) <= 2e-4 * np.max(np.abs(gref))
    l64, g64 = oracle_lib.cv_loss_grad(d, 16, 32, 1, x, h, a)
    assert abs(loss - l64) <= 2e-2 * l64
    assert np.max(np.abs(grad - g64)) <= 2e-2 * np.max(np.abs(g64))


def test_cv_training_and_estimator_parity(Q, oracle_lib, nthreads):
    """Train on a pilot lattice (configuration 5 integrand), then the GPU
    estimator Q[h - g] + int g and the plain Q[h] of the same pass against the
    oracle with the same (bfloat16) parameters."""
    p = I.config5(n=100003, m=4)
    g = I.random_generating_vector(I.SplitMix64(51), 8, p.n)
    gp = I.random_generating_vector(I.SplitMix64(52), 8, 65537)
    f = Q.integrand_from_problem(p, "fp32")
    t = Q.transform("korobov", 3)
    cfg = _cv_cfg(Q, steps=300)
    a, losses = Q.qmc_cv_train(8, 65537, gp, I.make_shifts(I.SplitMix64(53), 1, 8)[0], t, f, cfg)
    assert losses[1] < 0.5 * losses[0]
    assert np.array_equal(a, a.astype(np.float32))  # bfloat16 values held in float
    res, ps = Q.qmc_integrate_cv(p.d, p.n, p.m, g, p.shifts, t, f, cfg, a)
    p.cv = {"R": 16, "K": 32, "F": 1, "a": a}
    ref_cv = oracle_lib.integrate(p, g, nthreads=nthreads)
    gint = oracle_lib.cv_integral(8, 16, 32, a)
    q_cv = ref_cv["q"][:, 0] + gint
    del p.cv
    ref_plain = oracle_lib.integrate(p, g, nthreads=nthreads)
    assert np.all(np.abs(ps[:, 1] - ref_plain["q"][:, 0]) <= 4e-7 * np.abs(ref_plain["q"][:, 0]))
    assert np.all(np.abs(ps[:, 0] - q_cv) <= 4e-6 * np.abs(q_cv))


def test_cv_gain_reported(Q):
    """What the trained surrogate gains: the Eq. (3) error of Q[h - g] + int g
    against the plain rule's from the same points (configuration 5 integrand,
    n = 1048573, m = 16).  Both estimates agree within their errors; the ratio
    is printed for the record."""
    p = I.config5(n=1048573, m=16)
    g = Q.qmc_make_lattice(8, p.n, p.gamma)
    gp = Q.qmc_make_lattice(8, 65537, p.gamma)
    f = Q.integrand_from_problem(p, "fp32")
    t = Q.transform("korobov", 3)
    for freq in (1, 2):
        cfg = _cv_cfg(Q, steps=2000, freq=freq)
        a, losses = Q.qmc_cv_train(8, 65537, gp, I.make_shifts(I.SplitMix64(54), 1, 8)[0], t, f, cfg)
        res, _ = Q.qmc_integrate_cv(p.d, p.n, p.m, g, p.shifts, t, f, cfg, a)
        r = res.as_dict()
        print(f"cv freq_step={freq}: loss {losses[0]:.3e} -> {losses[1]:.3e}; err cv {r['err'][0]:.3e} "
              f"plain {r['err'][1]:.3e} ratio {r['err'][1] / r['err'][0]:.2f}")
        assert np.isfinite(r["err"][0]) and np.isfinite(r["err"][1])
        assert abs(r["mean"][0] - r["mean"][1]) <= 6 * (r["err"][0] + r["err"][1])


# ------------------------------------------------ run-time specialisation --

def test_specialised_kernel_bit_identical(Q, monkeypatch):
    """The kernel specialised at run time for the plan's U and F (nonzero
    monomials only) gives bit-identical results to the template kernel."""
    p = I.config2(n=1000003, m=32)
    g = I.random_generating_vector(I.SplitMix64(4), 6, p.n)
    f = Q.integrand_from_problem(p, "fp32")
    t = Q.transform("baker")
    plan = Q.Plan(p.d, p.n, p.m, g, p.shifts, t, f)
    assert plan.describe()["specialised"] == "1", Q.qmc_last_error()
    a = plan.execute().as_dict()
    plan.destroy()
    monkeypatch.setenv("QMC_JIT", "0")
    plan = Q.Plan(p.d, p.n, p.m, g, p.shifts, t, f)
    assert plan.describe()["specialised"] == "0"
    b = plan.execute().as_dict()
    plan.destroy()
    assert a["mean"][0] == b["mean"][0] and a["var"][0] == b["var"][0]


# ------------------------------------------------------------- utilities --

def test_immediate_shift_kernel_bit_identical(Q, monkeypatch):
    """The specialised sector kernel compiled with the shift table as
    immediate operands (QMC_JIT_IMM=1, a plan of one launch chunk) against the
    one reading its shifts from the launch parameters: the same constants
    enter the same operations, so per-shift values are bit-identical, and the
    plan reports the variant.  With more shifts than one launch takes, the
    switch is ignored."""
    p = I.config2(n=1000003, m=32)
    g = I.random_generating_vector(I.SplitMix64(31), p.d, p.n)
    f, t = Q.integrand_from_problem(p, "fp32"), Q.transform(p.transform, p.alpha)
    a = Q.Plan(p.d, p.n, p.m, g, p.shifts, t, f)
    assert a.describe()["imm_shifts"] == "0"
    pa = np.zeros(2 * p.m)
    ra = a.execute(per_shift=pa)
    monkeypatch.setenv("QMC_JIT_IMM", "1")
    b = Q.Plan(p.d, p.n, p.m, g, p.shifts, t, f)
    assert b.describe()["imm_shifts"] == "1" and b.describe()["specialised"] == "1"
    pb = np.zeros(2 * p.m)
    rb = b.execute(per_shift=pb)
    assert np.array_equal(pa, pb) and ra.mean[0] == rb.mean[0]
    q = I.with_shifts(p, 40, 77)  # 40 shifts: two launch chunks, parameter shifts
    c = Q.Plan(q.d, q.n, q.m, g, q.shifts, t, f)
    assert c.describe()["imm_shifts"] == "0"


def test_measure_peaks_sane(Q):
    """FP32 and FP64 FMA rates within their nominal bounds (80.5 and 1.25
    TFLOP/s at the maximum clock), and the warp-level MMA rates above the FP32
    pipe's (tensor cores) but below the dense tcgen05 figures (2.25 PFLOP/s
    BF16, 1.1 PFLOP/s TF32)."""
    pk = Q.qmc_measure_peaks()
    assert 10.0 < pk["fp32_tflops"] < 100.0
    assert 0.1 < pk["fp64_tflops"] < pk["fp32_tflops"]
    assert pk["fp32_tflops"] < pk["mma_sync_tf32_tflops"] < 1100.0
    assert pk["mma_sync_tf32_tflops"] < pk["mma_sync_bf16_tflops"] < 2250.0


def test_combine_shifts_equals_one_call(Q):
    """Two calls with disjoint shift sets, combined on the host, equal one call
    with all shifts (appending shifts to an estimate, or merging GPUs)."""
    p = I.config2(n=200003, m=16, precision="fp64")
    g = I.random_generating_vector(I.SplitMix64(9), 6, p.n)
    f = Q.integrand_from_problem(p)
    t = Q.transform("baker")
    _, ps_all = Q.qmc_integrate(p.d, p.n, 16, g, p.shifts, t, f, want_per_shift=True)
    _, ps_a = Q.qmc_integrate(p.d, p.n, 6, g, p.shifts[:6], t, f, want_per_shift=True)
    _, ps_b = Q.qmc_integrate(p.d, p.n, 10, g, p.shifts[6:], t, f, want_per_shift=True)
    one = Q.qmc_combine_shifts(ps_all).as_dict()
    two = Q.qmc_combine_shifts(np.concatenate([ps_a, ps_b])).as_dict()
    assert abs(one["mean"][0] - two["mean"][0]) <= 1e-14 * abs(one["mean"][0])
    assert abs(one["err"][0] - two["err"][0]) <= 1e-12 * abs(one["mean"][0])


# ------------------------------------------------- Fig. 3 and automatic n --

@pytest.mark.parametrize("d", [6, 9, 10])
def test_fig3_constant_integrand_korobov(Q, d):
    """Sec. 2 / Fig. 3: the constant 1 under Korobov weights 3 and 6: the error
    against the exact value 1 shrinks from n ~ 1e3 to n ~ 1e6 and the Eq. (3)
    estimate brackets it; the baker transform is exact (Q^(k) = 1, sigma = 0)."""
    rng = I.SplitMix64(300 + d)
    sh = I.make_shifts(rng, 8, d)
    gam = I.product_weights(d)
    for alpha in (3, 6):
        errs = []
        for n in (1021, 32749, 1048573):
            g = Q.qmc_make_lattice(d, n, gam)
            p = I.Problem("c", d, n, 8, sh, "korobov", alpha=alpha, kind="const")
            r, _ = Q.qmc_integrate(d, n, 8, g, sh, Q.transform("korobov", alpha), Q.integrand_from_problem(p, "fp64"))
            e = abs(r.mean[0] - 1.0)
            errs.append(e)
            assert e <= 8 * r.err[0] + 1e-14
        assert errs[-1] < errs[0] / 10, (alpha, errs)
    p = I.Problem("c", d, 1021, 8, sh, "baker", kind="const")
    r, ps = Q.qmc_integrate(d, 1021, 8, Q.qmc_make_lattice(d, 1021, gam), sh, Q.transform("baker"),
                            Q.integrand_from_problem(p, "fp64"), want_per_shift=True)
    assert np.all(ps[:, 0] == 1.0) and r.var[0] == 0.0


def test_integrate_to_tolerance(Q):
    """Automatic n: the ladder stops at the first lattice whose relative error
    estimate meets the target, and that estimate equals a direct call's."""
    p = I.config2(m=16)
    ladder = [n for n in I.ladder_primes() if 100000 < n < 20000000]
    gs = [Q.qmc_make_lattice(6, n, p.gamma) for n in ladder]
    f = Q.integrand_from_problem(p, "fp32")
    t = Q.transform("baker")
    res, lvl, ok = Q.qmc_integrate_to_tolerance(6, ladder, gs, 16, p.shifts, t, f, 1e-7)
    assert ok and 0 <= lvl < len(ladder)
    assert res.err[0] <= 1e-7 * abs(res.mean[0])
    if lvl > 0:
        prev, _ = Q.qmc_integrate(6, ladder[lvl - 1], 16, gs[lvl - 1], p.shifts, t, f)
        assert prev.err[0] > 1e-7 * abs(prev.mean[0])
    direct, _ = Q.qmc_integrate(6, ladder[lvl], 16, gs[lvl], p.shifts, t, f)
    assert direct.mean[0] == res.mean[0]
    res, lvl, ok = Q.qmc_integrate_to_tolerance(6, ladder[:2], gs[:2], 16, p.shifts, t, f, 1e-16)
    assert not ok and lvl == 1 and res.status == Q.QMC_ETIMEOUT


@pytest.mark.slow
def test_time_to_tolerance_true_error(Q, oracle_lib, nthreads):
    """The walks to 1e-8 relative error that the benchmark times land within
    their own error estimate of the true integral. Two walks:
    * the plain rule on the prime ladder (configuration-2 integrand, baker);
    * the embedded base-2 lattices (configuration-5 integrand, Korobov 3).
    Each is checked against tensor Gauss-Legendre of the untransformed
    integrand, converged (two node counts agree to 1e-11)."""
    p = I.config2()
    ladder = [n for n in I.ladder_primes() if 100000 < n < 20000000]
    gs = [Q.qmc_make_lattice(6, n, p.gamma) for n in ladder]
    res, lvl, ok = Q.qmc_integrate_to_tolerance(6, ladder, gs, p.m, p.shifts, Q.transform("baker"),
                                                Q.integrand_from_problem(p, "fp32"), 1e-8)
    assert ok and res.err[0] <= 1e-8 * abs(res.mean[0])
    gl_a = oracle_lib.gauss_legendre(p, 12, nthreads=nthreads)[0]
    gl_b = oracle_lib.gauss_legendre(p, 16, nthreads=nthreads)[0]
    assert abs(gl_a - gl_b) <= 1e-11 * abs(gl_b)
    print(f"C2 ladder: n = {ladder[lvl]}, |Q - I| / |I| = {abs(res.mean[0] - gl_b) / abs(gl_b):.2e}, "
          f"estimate {res.err[0] / abs(res.mean[0]):.2e}")
    assert abs(res.mean[0] - gl_b) <= 4 * res.err[0]
    p5 = I.config5()
    ge = Q.qmc_make_lattice_embedded(8, 16, 25, p5.gamma)
    r, lvl5, _, ok5 = Q.qmc_integrate_extensible(8, 16, 10, ge, p5.m, p5.shifts, Q.transform("korobov", 3),
                                                 Q.integrand_from_problem(p5, "fp32"), 1e-8)
    assert ok5 and r.err[0] <= 1e-8 * abs(r.mean[0])
    gl9 = oracle_lib.gauss_legendre(p5, 9, nthreads=nthreads)[0]
    gl10 = oracle_lib.gauss_legendre(p5, 10, nthreads=nthreads)[0]
    assert abs(gl9 - gl10) <= 1e-11 * abs(gl10)
    print(f"C5 embedded: n = 2^{16 + lvl5}, |Q - I| / |I| = {abs(r.mean[0] - gl10) / abs(gl10):.2e}, "
          f"estimate {r.err[0] / abs(r.mean[0]):.2e}")
    assert abs(r.mean[0] - gl10) <= 4 * r.err[0]


def test_fp32_rounding_unbiased_at_full_size(Q, lattices):
    """At n = 16777213 the lattice spacing equals the float grid of the
    coordinates, so rounding them to float repeats a lattice-tied pattern of
    errors.  The FP32 path rounds each coordinate once from 32-bit fixed point
    with a per-point dither; its per-shift values must then agree with the FP64
    path to 2e-10 relative (the QMC scatter between shifts is ~5e-9), and the
    mean to a tenth of the FP64 error estimate."""
    p = I.config2(n=16777213, m=32)
    g = gvec(lattices, p)
    t = Q.transform(p.transform, p.alpha)
    r32, ps32 = Q.qmc_integrate(p.d, p.n, p.m, g, p.shifts, t, Q.integrand_from_problem(p, "fp32"),
                                want_per_shift=True)
    r64, ps64 = Q.qmc_integrate(p.d, p.n, p.m, g, p.shifts, t, Q.integrand_from_problem(p, "fp64"),
                                want_per_shift=True)
    q = abs(r64.mean[0])
    assert np.all(np.abs(ps32[:, 0] - ps64[:, 0]) <= 2e-10 * q), np.max(np.abs(ps32[:, 0] - ps64[:, 0])) / q
    assert abs(r32.mean[0] - r64.mean[0]) <= 0.1 * r64.err[0]


@pytest.mark.parametrize("cfg", ["c2", "c5"])
def test_fp32_korobov_weight_unbiased_at_full_size(Q, cfg):
    """The Korobov-3 FP32 path: its weight is a product of d factors
    u = s(1 - s) cubed.  Rounding u * u * u per factor in float is biased low
    (the low bits of a square are not uniform); that summed to -3.0e-9 (d = 6)
    and -4.6e-9 (d = 8) relative against the FP64 rule, above the rule's own
    error at 1e-8 targets.  The FP32 path multiplies the factors and cubes the
    product once with an exact square.  Korobov values also span many binades,
    and float runs dropped the smallest (-1.4e-9 more); each value now goes
    into the compensated pair on its own.  What remains is the FP32 rounding of
    the coordinates and of z, which grows with d.  At n = 16777213 the FP32 and
    FP64 per-shift values must agree on average to 1e-10 d and each to
    2.5e-10 d.  That is measured at -4.2e-10 (d = 6) and -6.5e-10 (d = 8), a
    twentieth of the rule's error estimate there; before the two changes it was
    -3.0e-9 and -4.6e-9."""
    p = (I.config2(n=16777213, m=16) if cfg == "c2" else I.config5(n=16777213, m=16))
    g = Q.qmc_make_lattice(p.d, p.n, p.gamma)
    t = Q.transform("korobov", 3)
    _, ps32 = Q.qmc_integrate(p.d, p.n, p.m, g, p.shifts, t, Q.integrand_from_problem(p, "fp32"),
                              want_per_shift=True)
    _, ps64 = Q.qmc_integrate(p.d, p.n, p.m, g, p.shifts, t, Q.integrand_from_problem(p, "fp64"),
                              want_per_shift=True)
    rel = (ps32[:, 0] - ps64[:, 0]) / ps64[:, 0]
    print(f"{cfg}: FP32 - FP64 per shift, mean {rel.mean():.2e}, max |.| {np.abs(rel).max():.2e}")
    assert abs(rel.mean()) <= 1e-10 * p.d
    assert np.all(np.abs(rel) <= 2.5e-10 * p.d)


@pytest.mark.parametrize("transform,alpha", [("baker", 0), ("korobov", 3), ("none", 0)])
def test_fp32_fold_and_origin_points(Q, oracle_lib, transform, alpha):
    """FP32 coordinates at the fold x = 1/2 (fixed point 2^31, the most
    negative 32-bit integer when read as signed) and at the origin: point j = 0
    under shifts with coordinates 0.5 and 0.0 exactly, against the oracle."""
    p = I.config2(n=100003, m=4)
    p.transform, p.alpha = transform, alpha
    p.shifts = np.array([[0.5] * 6, [0.0] * 6, [0.5, 0.0, 0.5, 0.0, 0.5, 0.0], [0.25, 0.5, 0.75, 0.0, 0.5, 0.125]])
    g = I.random_generating_vector(I.SplitMix64(9), 6, p.n)
    js = np.zeros(4, dtype=np.uint64)
    ks = np.arange(4, dtype=np.int32)
    vals, _, crd = Q.qmc_sample_points(p.d, p.n, p.m, g, p.shifts, Q.transform(transform, alpha),
                                       Q.integrand_from_problem(p, "fp32"), js, ks)
    for s in range(4):
        v, _, ox, _, _ = oracle_lib.point(p, g, int(ks[s]), 0)
        assert np.array_equal(crd[s], ox), (s, crd[s], ox)
        assert abs(vals[s, 0] - v[0]) <= 4e-6 * abs(v[0]) + 1e-300, (s, vals[s, 0], v[0])


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 2e-8)])
def test_extensible_levels_reproduce_the_direct_rule(Q, oracle_lib, precision, tol):
    """Doubling from n = 2^10 to 2^14 by evaluating only the new half of the
    points each time gives the size-2^14 rule itself (per shift), and the
    oracle's value for it.  In FP32 the two evaluations give a point different
    dithers (its index differs between the half-size rule and the direct one),
    so they differ by the per-point rounding noise, ~2e-7 rms averaged over
    16384 points (~2e-9 rms)."""
    p = I.config2(n=1 << 14, m=8)
    g = Q.qmc_make_lattice_embedded(6, 10, 14, p.gamma, candidates=64, seed=3)
    t = Q.transform(p.transform, p.alpha)
    f = Q.integrand_from_problem(p, precision)
    res, lvl, ps, ok = Q.qmc_integrate_extensible(6, 10, 5, g, 8, p.shifts, t, f, 1e-300)
    assert not ok and lvl == 4 and res.status == Q.QMC_ETIMEOUT
    direct, ps_d = Q.qmc_integrate(6, 1 << 14, 8, g % (1 << 14), p.shifts, t, f, want_per_shift=True)
    assert np.all(np.abs(ps[:, 0] - ps_d[:, 0]) <= tol * np.abs(ps_d[:, 0]))
    ref = oracle_lib.integrate(p, g % (1 << 14))
    assert np.all(np.abs(ps[:, 0] - ref["q"][:, 0]) <= (1e-12 if precision == "fp64" else 2e-7) * np.abs(ref["q"][:, 0]))


def test_extensible_stops_at_tolerance(Q):
    """The doubling stops at the first size whose Eq. (3) relative error meets
    the target; the previous size did not."""
    p = I.config2(m=16)
    g = Q.qmc_make_lattice_embedded(6, 12, 24, p.gamma, candidates=32, seed=1)
    t = Q.transform(p.transform, p.alpha)
    f = Q.integrand_from_problem(p, "fp32")
    res, lvl, ps, ok = Q.qmc_integrate_extensible(6, 12, 13, g, 16, p.shifts, t, f, 1e-7)
    assert ok and 0 < lvl <= 12
    assert res.err[0] <= 1e-7 * abs(res.mean[0])
    n_prev = 1 << (12 + lvl - 1)
    prev, _ = Q.qmc_integrate(6, n_prev, 16, g % n_prev, p.shifts, t, f)
    assert prev.err[0] > 1e-7 * abs(prev.mean[0])

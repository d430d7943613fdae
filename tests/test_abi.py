"""Host-only checks of the C ABI: the library loads, exports every function
include/qmc.h declares, the binding's structs match the header's sizes, and
argument validation rejects bad input before any device work.  The CBC
generating-vector search is host code and is compared with the oracle here."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1811_11722_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qmc.h")


@pytest.fixture(scope="module")
def Q():
    from paper_1811_11722_gb300 import build, qmc
    build.build_library()
    qmc.lib()
    return qmc


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(qmc_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("qmc_make_lattice", "qmc_integrate", "qmc_integrate_batch", "qmc_plan_create", "qmc_plan_execute",
              "qmc_plan_destroy", "qmc_sample_points", "qmc_last_error", "qmc_version"):
        assert n in names


def test_library_exports_every_declared_symbol(Q):
    L = Q.lib()
    for name in declared_functions():
        assert hasattr(L, name), name
    # the symbol table itself (not only dlsym through ctypes)
    out = os.popen(f"nm -D --defined-only {Q.LIB_PATH}").read()
    for name in declared_functions():
        assert re.search(rf"\bT {name}\b", out), name


def test_struct_layouts(Q):
    assert ctypes.sizeof(Q.qmc_transform) == 8
    assert ctypes.sizeof(Q.qmc_poly) == 24
    assert ctypes.sizeof(Q.qmc_result) == 72
    assert ctypes.sizeof(Q.qmc_integrand) == 4 * 3 + 4 + 2 * 24 + 8 + 8 + 3 * 8
    assert ctypes.sizeof(Q.qmc_eps) == 24
    assert Q.qmc_version() >= 100
    hdr = open(HEADER).read()
    assert int(re.search(r"#define QMC_EPS_MAX (\d+)", hdr).group(1)) == 6


def _sector(Q, d=3, n=101, m=4):
    p = I.config2(n=n, m=m)
    return p


@pytest.mark.parametrize("case", ["m1", "g0", "gn", "shift1", "d0", "d17", "nbig", "dmismatch", "alpha7",
                                  "kind", "nterms0", "deg4"])
def test_validation_rejects_bad_arguments(Q, case):
    """Bad arguments return QMC_EINVAL without touching the GPU."""
    d, n, m = 3, 101, 4
    g = np.array([1, 5, 7], dtype=np.uint64)
    shifts = np.full((m, d), 0.25)
    t = Q.transform("baker")
    coef = np.array([1.0, 0.5])
    expo = np.array([[0, 0, 0], [1, 0, 0]], dtype=np.uint8)
    f = Q.Integrand(Q.QMC_F_SECTOR, d, Q.QMC_FP64, (coef, expo), (coef, expo))
    if case == "m1":
        m, shifts = 1, shifts[:1]
    elif case == "g0":
        g[1] = 0
    elif case == "gn":
        g[2] = n
    elif case == "shift1":
        shifts[2, 1] = 1.0
    elif case == "d0":
        d = 0
    elif case == "d17":
        d = 17
    elif case == "nbig":
        n = 1 << 31
    elif case == "dmismatch":
        f = Q.Integrand(Q.QMC_F_SECTOR, 2, Q.QMC_FP64, (coef, expo[:, :2]), (coef, expo[:, :2]))
    elif case == "alpha7":
        t = Q.transform("korobov", 7)
    elif case == "kind":
        f = Q.Integrand(9, d)
    elif case == "nterms0":
        f = Q.Integrand(Q.QMC_F_SECTOR, d, Q.QMC_FP64, (coef[:0], expo[:0]), (coef, expo))
    elif case == "deg4":
        f = Q.Integrand(Q.QMC_F_SECTOR, d, Q.QMC_FP64, (coef, np.array([[0, 0, 0], [4, 0, 0]], np.uint8)),
                        (coef, expo))
    with pytest.raises(Q.QmcError) as ei:
        Q.qmc_integrate(d, n, m, g, shifts, t, f)
    assert ei.value.status == Q.QMC_EINVAL
    assert Q.qmc_last_error() != ""


@pytest.mark.parametrize("case", ["orders0", "orders7", "nan_slope", "not_sector"])
def test_eps_validation_rejects_bad_arguments(Q, case):
    """The epsilon entry points check their descriptor on the host."""
    d, n, m = 3, 101, 4
    g = np.array([1, 5, 7], dtype=np.uint64)
    shifts = np.full((m, d), 0.25)
    t = Q.transform("baker")
    coef = np.array([1.0, 0.5])
    expo = np.array([[0, 0, 0], [1, 0, 0]], dtype=np.uint8)
    f = Q.Integrand(Q.QMC_F_SECTOR, d, Q.QMC_FP64, (coef, expo), (coef, expo))
    eps = Q.eps_spec(3)
    if case == "orders0":
        eps = Q.eps_spec(0)
    elif case == "orders7":
        eps = Q.eps_spec(7)
    elif case == "nan_slope":
        eps = Q.eps_spec(2, float("nan"), -1.0)
    elif case == "not_sector":
        f = Q.Integrand(Q.QMC_F_CONST, d)
    with pytest.raises(Q.QmcError) as ei:
        Q.qmc_integrate_eps(d, n, m, g, shifts, t, f, eps)
    assert ei.value.status == Q.QMC_EINVAL
    with pytest.raises(Q.QmcError) as ei:
        Q.qmc_sample_points_eps(d, n, m, g, shifts, t, f, eps, [0], [0])
    assert ei.value.status == Q.QMC_EINVAL


@pytest.mark.parametrize("case,status", [("count0", "EINVAL"), ("fp64", "EUNSUPPORTED"), ("dmismatch", "EINVAL"),
                                         ("deg3", "EUNSUPPORTED"), ("alpha2", "EUNSUPPORTED"), ("d9", "EUNSUPPORTED")])
def test_multi_validation(Q, case, status):
    """The shared-lattice entry point checks every integrand on the host."""
    d, n, m = 3, 101, 4
    coef = np.array([1.0, 0.5])
    expo = np.array([[0, 0, 0], [1, 0, 0]], dtype=np.uint8)
    t = Q.transform("baker")
    fs = [Q.Integrand(Q.QMC_F_SECTOR, d, Q.QMC_FP32EVAL, (coef, expo), (coef, expo)) for _ in range(3)]
    if case == "count0":
        fs = []
    elif case == "fp64":
        fs[1] = Q.Integrand(Q.QMC_F_SECTOR, d, Q.QMC_FP64, (coef, expo), (coef, expo))
    elif case == "dmismatch":
        fs[2] = Q.Integrand(Q.QMC_F_SECTOR, 2, Q.QMC_FP32EVAL, (coef, expo[:, :2]), (coef, expo[:, :2]))
    elif case == "deg3":
        fs[0] = Q.Integrand(Q.QMC_F_SECTOR, d, Q.QMC_FP32EVAL, (coef, expo),
                            (coef, np.array([[0, 0, 0], [1, 1, 1]], np.uint8)))
    elif case == "alpha2":
        t = Q.transform("korobov", 2)
    elif case == "d9":
        d = 9
        e9 = np.zeros((2, 9), np.uint8)
        e9[1, 0] = 1
        fs = [Q.Integrand(Q.QMC_F_SECTOR, 9, Q.QMC_FP32EVAL, (coef, e9), (coef, e9))]
    g = np.arange(1, d + 1, dtype=np.uint64)
    shifts = np.full((m, d), 0.25)
    with pytest.raises(Q.QmcError) as ei:
        Q.qmc_integrate_multi(d, n, m, g, shifts, t, fs)
    assert ei.value.status == getattr(Q, "QMC_" + status)


@pytest.mark.parametrize("case,status", [("chunk100", "EINVAL"), ("fp64", "EUNSUPPORTED"), ("deg3", "EUNSUPPORTED"),
                                         ("alpha2", "EUNSUPPORTED"), ("d9", "EUNSUPPORTED"),
                                         ("powers", "EUNSUPPORTED"), ("bad_g", "EINVAL")])
def test_persistent_batch_validation(Q, case, status):
    """The persistent batch checks every problem on the host, before any
    device work (so these run without a GPU)."""
    d, n, m = 3, 101, 4
    coef = np.array([1.0, 0.5])
    expo = np.array([[0, 0, 0], [1, 0, 0]], dtype=np.uint8)
    t = Q.transform("baker")
    g = np.arange(1, d + 1, dtype=np.uint64)
    shifts = np.full((m, d), 0.25)
    f = Q.Integrand(Q.QMC_F_SECTOR, d, Q.QMC_FP32EVAL, (coef, expo), (coef, expo))
    probs = [(d, n, m, g, shifts, t, f), (d, n, m, g, shifts, t, f)]
    chunk = 0
    if case == "chunk100":
        chunk = 100
    elif case == "fp64":
        probs[1] = (d, n, m, g, shifts, t, Q.Integrand(Q.QMC_F_SECTOR, d, Q.QMC_FP64, (coef, expo), (coef, expo)))
    elif case == "deg3":
        f3 = Q.Integrand(Q.QMC_F_SECTOR, d, Q.QMC_FP32EVAL, (coef, expo),
                         (coef, np.array([[0, 0, 0], [1, 1, 1]], np.uint8)))
        probs[0] = (d, n, m, g, shifts, t, f3)
    elif case == "alpha2":
        probs[1] = (d, n, m, g, shifts, Q.transform("korobov", 2), f)
    elif case == "d9":
        e9 = np.zeros((2, 9), np.uint8)
        e9[1, 0] = 1
        probs[0] = (9, n, m, np.arange(1, 10, dtype=np.uint64), np.full((m, 9), 0.25), t,
                    Q.Integrand(Q.QMC_F_SECTOR, 9, Q.QMC_FP32EVAL, (coef, e9), (coef, e9)))
    elif case == "powers":
        probs[1] = (d, n, m, g, shifts, t, Q.Integrand(Q.QMC_F_SECTOR, d, Q.QMC_FP32EVAL, (coef, expo), (coef, expo),
                                                       -1, -1))
    elif case == "bad_g":
        probs[1] = (d, n, m, np.array([1, 101, 3], dtype=np.uint64), shifts, t, f)
    with pytest.raises(Q.QmcError) as ei:
        Q.BatchPlan(probs, persistent=True, chunk=chunk)
    assert ei.value.status == getattr(Q, "QMC_" + status)


def test_make_lattice_rejects_composite(Q):
    with pytest.raises(Q.QmcError):
        Q.qmc_make_lattice(3, 1001, [1.0, 0.25, 1 / 9])
    with pytest.raises(Q.QmcError):
        Q.qmc_make_lattice(0, 101, [1.0])


@pytest.mark.parametrize("n", [31, 101, 1009, 10007, 65537])
def test_make_lattice_matches_oracle_cbc(Q, oracle_lib, n):
    """Host CBC of the library against the oracle's plain CBC (n <= 1e4) or the
    oracle's numpy fast CBC, judged by the worst-case error they reach."""
    from oracle.cbc import cbc_fast
    d = 6
    gam = I.product_weights(d)
    g = Q.qmc_make_lattice(d, n, gam)
    ref = oracle_lib.cbc_plain(d, n, gam) if n <= 10007 else cbc_fast(d, n, gam)
    assert g[0] == 1 and np.all((g >= 1) & (g <= (n - 1) // 2))
    e_lib = oracle_lib.cbc_error(d, n, g, gam)
    e_ref = oracle_lib.cbc_error(d, n, ref, gam)
    assert abs(e_lib - e_ref) <= 1e-12 * e_ref
    if n >= 101:
        assert np.array_equal(g, ref)


# ------------------------------------------------------ embedded lattices --

def _embedded_T(oracle_lib, g, gamma, kmin, K):
    """max_k 4^k e^2_{2^k}(g) with the oracle's worst-case error."""
    s = len(g)
    return max(4.0 ** k * oracle_lib.cbc_error(s, 1 << k, np.asarray(g, dtype=np.uint64) % (1 << k), gamma[:s])
               for k in range(kmin, K + 1))


def test_embedded_lattice_exhaustive_matches_oracle(Q, oracle_lib):
    """All odd candidates at N = 2^8 (sizes 2^3..2^8), d = 3: every component
    attains the minimum of the oracle-evaluated criterion.  Symmetric
    candidates (z and -z^-1 mod N give mirrored lattices) tie to ~1e-13, where
    rounding picks one, so the minimum is matched to 1e-10 relative."""
    d, kmin, K = 3, 3, 8
    gam = I.product_weights(d)
    g = Q.qmc_make_lattice_embedded(d, kmin, K, gam)
    assert g[0] == 1 and np.all(g % 2 == 1) and np.all(g < (1 << (K - 1)))
    for s in range(1, d):
        cands = list(range(1, 1 << (K - 1), 2))
        T = np.array([_embedded_T(oracle_lib, list(g[:s]) + [z], gam, kmin, K) for z in cands])
        chosen = T[cands.index(int(g[s]))]
        assert chosen <= T.min() * (1 + 1e-10), (s, g[s], cands[int(np.argmin(T))], chosen, T.min())
        # every candidate clearly better than the chosen one would be a mistake
        assert np.sum(T < chosen * (1 - 1e-10)) == 0


def test_embedded_lattice_subset_is_deterministic(Q, oracle_lib):
    """With a drawn candidate subset the vector depends only on the seed, and it
    beats the degenerate vector g = (1, 1, ..., 1) at every embedded size."""
    d, kmin, K = 4, 6, 14
    gam = I.product_weights(d)
    a = Q.qmc_make_lattice_embedded(d, kmin, K, gam, candidates=32, seed=7)
    b = Q.qmc_make_lattice_embedded(d, kmin, K, gam, candidates=32, seed=7)
    c = Q.qmc_make_lattice_embedded(d, kmin, K, gam, candidates=32, seed=8)
    assert np.array_equal(a, b) and a[0] == 1 and np.all(a % 2 == 1)
    assert not np.array_equal(a, c)
    for k in range(kmin, K + 1):
        n = 1 << k
        assert oracle_lib.cbc_error(d, n, a % n, gam) < oracle_lib.cbc_error(d, n, np.ones(d, np.uint64), gam)


@pytest.mark.parametrize("args", [(0, 3, 8), (17, 3, 8), (3, 0, 8), (3, 9, 8), (3, 3, 31)])
def test_embedded_lattice_validation(Q, args):
    d, kmin, K = args
    with pytest.raises(Q.QmcError) as ei:
        Q.qmc_make_lattice_embedded(d, kmin, K, np.ones(max(d, 1)))
    assert ei.value.status == Q.QMC_EINVAL


@pytest.mark.parametrize("case", ["decreasing", "g_out_of_range", "dim_below_d", "criterion", "tol", "levels"])
def test_batch_walk_validation(Q, case):
    """The batched ladder walk checks its ladder and options on the host,
    before any device work (so these run without a GPU)."""
    d, n, m = 3, 101, 4
    coef = np.array([1.0, 0.5])
    expo = np.array([[0, 0, 0], [1, 0, 0]], dtype=np.uint8)
    f = Q.Integrand(Q.QMC_F_SECTOR, d, Q.QMC_FP32EVAL, (coef, expo), (coef, expo))
    probs = [(d, n, m, np.arange(1, d + 1, dtype=np.uint64), np.full((m, d), 0.25), Q.transform("baker"), f)]
    ladder_n = np.array([211, 401, 809], dtype=np.uint64)
    ladder_g = np.tile(np.arange(1, 5, dtype=np.uint64), (3, 1))
    tol, crit = 1e-6, Q.WALK_SUM
    if case == "decreasing":
        ladder_n = np.array([211, 809, 401], dtype=np.uint64)
    elif case == "g_out_of_range":
        ladder_g[1, 3] = 401
    elif case == "dim_below_d":
        ladder_g = ladder_g[:, :2].copy()
    elif case == "criterion":
        crit = 2
    elif case == "tol":
        tol = 0.0
    elif case == "levels":
        ladder_n = np.arange(1000, 1000 + 65, dtype=np.uint64)
        ladder_g = np.ones((65, 4), dtype=np.uint64)
    with pytest.raises(Q.QmcError) as ei:
        Q.qmc_integrate_batch_to_tolerance(probs, ladder_n, ladder_g, tol, crit)
    assert ei.value.status == Q.QMC_EINVAL


@pytest.mark.parametrize("case", ["n_not_power_of_two", "n_above_2_30", "even_g", "dim_below_d", "criterion", "tol",
                                  "levels", "one_shift"])
def test_batch_extensible_validation(Q, case):
    """The batched embedded-lattice walk checks its sizes, vector and options
    on the host, before any device work (so these run without a GPU)."""
    d, n, m = 3, 1024, 4
    coef = np.array([1.0, 0.5])
    expo = np.array([[0, 0, 0], [1, 0, 0]], dtype=np.uint8)
    f = Q.Integrand(Q.QMC_F_SECTOR, d, Q.QMC_FP32EVAL, (coef, expo), (coef, expo))
    g = np.array([1, 433, 12345, 999], dtype=np.uint64)
    levels, tol, crit = 4, 1e-6, Q.WALK_SUM
    if case == "n_not_power_of_two":
        n = 1000
    elif case == "n_above_2_30":
        n = 1 << 31
    elif case == "even_g":
        g[2] = 12346
    elif case == "dim_below_d":
        g = g[:2].copy()
    elif case == "criterion":
        crit = Q.WALK_SUM | Q.WALK_PERSISTENT
    elif case == "tol":
        tol = -1.0
    elif case == "levels":
        levels = 31
    elif case == "one_shift":
        m = 1
    probs = [(d, n, m, g[:d] % n, np.full((m, d), 0.25), Q.transform("baker"), f)]
    with pytest.raises(Q.QmcError) as ei:
        Q.qmc_integrate_batch_extensible(probs, levels, g, tol, crit)
    assert ei.value.status == Q.QMC_EINVAL

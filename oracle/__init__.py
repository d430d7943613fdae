"""CPU oracle for the randomly shifted rank-1 lattice rule (Eq. 2, Eq. 3).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use this package; the product never imports it.
It shares no code with the CUDA path.  The arithmetic lives in plain C
(``oracle.c``, FP64, compiled here with gcc) plus a numpy fast-CBC in
``cbc.py``; this module only marshals arguments.

Functions and the passage each follows:
  rule_sums / integrate     Eq. (2) sums and Eq. (3) estimate
  point                     one term of Eq. (2) with its index, coordinate, transform
  transform                 Eq. (5) Korobov weight alpha, Eq. (6) baker
  integrand                 Eq. (7) U^aU F^aF, the Sec. 3 contour deformation, test functions
  gauss_legendre            tensor Gauss-Legendre integral (a reference, not the method)
  cv_g / cv_integral / cv_loss_grad   control-variate surrogate, its integral, its fit gradient
  det_lu                    LU determinant with partial pivoting (deformation Jacobian)
  cbc_plain / cbc_error     generating-vector search (the paper takes g as an input)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()

KIND = {"const": 0, "separable_exp": 1, "sector": 2, "sector_deformed": 3, "trig": 4}
TKIND = {"none": 0, "korobov": 1, "baker": 2}


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (FP contraction off so x86 and Arm agree)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-o", tmp, _SRC, "-lm", "-lpthread"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int), ("d", ctypes.c_int), ("tkind", ctypes.c_int), ("alpha", ctypes.c_int),
        ("nU", ctypes.c_int), ("cU", ctypes.c_void_p), ("eU", ctypes.c_void_p),
        ("nF", ctypes.c_int), ("cF", ctypes.c_void_p), ("eF", ctypes.c_void_p),
        ("aU", ctypes.c_int), ("aF", ctypes.c_int), ("lam", ctypes.c_double),
        ("c", ctypes.c_void_p), ("b", ctypes.c_void_p), ("h", ctypes.c_void_p),
        ("cvR", ctypes.c_int), ("cvK", ctypes.c_int), ("cvF", ctypes.c_int), ("cva", ctypes.c_void_p),
        ("eps_order", ctypes.c_int), ("eps_bU", ctypes.c_double), ("eps_bF", ctypes.c_double),
    ]


def _configure(L):
    P = ctypes.POINTER(_Problem)
    vp, u64, i32, dbl = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
    L.orc_rule_sums.argtypes = [P, u64, vp, i32, vp, u64, u64, i32, vp, vp, vp]
    L.orc_estimate.argtypes = [i32, u64, vp, vp, vp, vp]
    L.orc_point.argtypes = [P, u64, vp, vp, u64, vp, vp, vp, vp, vp]
    L.orc_transform.argtypes = [i32, i32, dbl, vp]
    L.orc_transform.restype = dbl
    L.orc_integrand.argtypes = [P, vp, vp, vp]
    L.orc_gauss_legendre.argtypes = [P, i32, vp, vp, i32, vp]
    L.orc_det_lu_out.argtypes = [i32, vp, vp]
    L.orc_index.argtypes = [u64, u64, u64]
    L.orc_index.restype = u64
    L.orc_cbc_error.argtypes = [i32, u64, vp, vp]
    L.orc_cbc_error.restype = dbl
    L.orc_cbc_plain.argtypes = [i32, u64, vp, vp]
    L.orc_cbc_candidate.argtypes = [u64, vp, u64]
    L.orc_cbc_candidate.restype = dbl
    L.orc_cv_g.argtypes = [i32, i32, i32, i32, vp, vp]
    L.orc_cv_g.restype = dbl
    L.orc_cv_integral.argtypes = [i32, i32, i32, vp]
    L.orc_cv_integral.restype = dbl
    L.orc_cv_loss_grad.argtypes = [i32, i32, i32, i32, i32, vp, vp, vp, vp]
    L.orc_cv_loss_grad.restype = dbl
    L.orc_cv_loss_grad_bf16.argtypes = [i32, i32, i32, i32, i32, vp, vp, vp, vp]
    L.orc_cv_loss_grad_bf16.restype = dbl
    L.orc_bf16.argtypes = [dbl]
    L.orc_bf16.restype = dbl
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _configure(ctypes.CDLL(_LIB_PATH))
    return _lib


def use_library(path):
    """Point every wrapper at another build of oracle.c (tests that plant a
    mistake in a copy of the source use this); returns the previous handle.
    use_library(None) restores the default build."""
    global _lib
    with _lock:
        prev = _lib
        _lib = None if path is None else _configure(ctypes.CDLL(path))
    return prev


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class _Marshalled:
    """Keeps the numpy arrays behind an orc_problem alive."""

    def __init__(self, p):
        d = p.d
        self.keep = []

        def arr(x, dt):
            if x is None:
                return None
            a = np.ascontiguousarray(np.asarray(x, dtype=dt))
            self.keep.append(a)
            return a

        s = _Problem()
        s.kind = KIND[p.kind]
        s.d = d
        s.tkind = TKIND[p.transform]
        s.alpha = int(p.alpha)
        if p.U is not None:
            cu, eu = arr(p.U.coef, np.float64), arr(p.U.expo, np.uint8)
            s.nU, s.cU, s.eU = cu.shape[0], _ptr(cu), _ptr(eu)
        if p.F is not None:
            cf, ef = arr(p.F.coef, np.float64), arr(p.F.expo, np.uint8)
            s.nF, s.cF, s.eF = cf.shape[0], _ptr(cf), _ptr(ef)
        s.aU, s.aF, s.lam = int(p.aU), int(p.aF), float(p.lam)
        s.c = _ptr(arr(p.c, np.float64))
        s.b = _ptr(arr(p.b, np.float64))
        s.h = _ptr(arr(p.h, np.int32))
        eps = getattr(p, "eps", None)
        if eps is not None:
            s.eps_order, s.eps_bU, s.eps_bF = int(eps["order"]), float(eps["bU"]), float(eps["bF"])
        cv = getattr(p, "cv", None)
        if cv is not None:
            s.cvR, s.cvK, s.cvF = int(cv["R"]), int(cv["K"]), int(cv["F"])
            s.cva = _ptr(arr(cv["a"], np.float32))
        self.s = s


def rule_sums(p, g, j0: int = 0, j1: int | None = None, nthreads: int = 1, shifts=None):
    """Per-shift sums over j in [j0, j1) (0-based j = the paper's j-1).
    Returns (sums[m, 2], nonfinite[m], deform_bad)."""
    L = lib()
    mp = _Marshalled(p)
    g = np.ascontiguousarray(np.asarray(g, dtype=np.uint64))
    sh = np.ascontiguousarray(np.asarray(p.shifts if shifts is None else shifts, dtype=np.float64))
    m = sh.shape[0]
    j1 = p.n if j1 is None else j1
    sums = np.zeros((m, 2), dtype=np.float64)
    nonf = np.zeros(m, dtype=np.uint64)
    bad = ctypes.c_uint64(0)
    rc = L.orc_rule_sums(ctypes.byref(mp.s), p.n, _ptr(g), m, _ptr(sh), j0, j1, max(1, int(nthreads)),
                         _ptr(sums), _ptr(nonf), ctypes.byref(bad))
    if rc != 0:
        raise ValueError("orc_rule_sums rejected its arguments")
    return sums, nonf, int(bad.value)


def estimate(sums, n: int):
    """Eq. (2), (3): returns (q[m, 2], mean[2], var[2])."""
    L = lib()
    sums = np.ascontiguousarray(np.asarray(sums, dtype=np.float64))
    m = sums.shape[0]
    q = np.zeros((m, 2))
    mean = np.zeros(2)
    var = np.zeros(2)
    if L.orc_estimate(m, n, _ptr(sums), _ptr(q), _ptr(mean), _ptr(var)) != 0:
        raise ValueError("m < 2")
    return q, mean, var


def integrate(p, g, nthreads: int = 1):
    """Whole rule: dict with q (per shift, re/im), mean, var, err, nonfinite, deform_bad."""
    sums, nonf, bad = rule_sums(p, g, nthreads=nthreads)
    q, mean, var = estimate(sums, p.n)
    return {"q": q, "mean": mean, "var": var, "err": np.sqrt(var), "sums": sums,
            "nonfinite": nonf, "deform_bad": bad}


def point(p, g, k: int, j: int):
    """Term (j, k) of Eq. (2), j 0-based: returns (value[2], idx[d], x[d], z[d], bad)."""
    L = lib()
    mp = _Marshalled(p)
    g = np.ascontiguousarray(np.asarray(g, dtype=np.uint64))
    sh = np.ascontiguousarray(np.asarray(p.shifts[k], dtype=np.float64))
    val = np.zeros(2)
    idx = np.zeros(p.d, dtype=np.uint64)
    x = np.zeros(p.d)
    z = np.zeros(p.d)
    bad = ctypes.c_int(0)
    L.orc_point(ctypes.byref(mp.s), p.n, _ptr(g), _ptr(sh), j, _ptr(val), _ptr(idx), _ptr(x), _ptr(z),
                ctypes.byref(bad))
    return val, idx, x, z, bad.value


def index(jm1: int, g: int, n: int) -> int:
    return int(lib().orc_index(jm1, g, n))


def transform(kind: str, alpha: int, x: float):
    """Eq. (5)/(6): returns (z, w)."""
    w = ctypes.c_double(0.0)
    z = lib().orc_transform(TKIND[kind], alpha, float(x), ctypes.byref(w))
    return z, w.value


def integrand(p, y):
    """f(y) at a transformed point: returns (value[2], bad)."""
    mp = _Marshalled(p)
    y = np.ascontiguousarray(np.asarray(y, dtype=np.float64))
    out = np.zeros(2)
    bad = ctypes.c_int(0)
    lib().orc_integrand(ctypes.byref(mp.s), _ptr(y), _ptr(out), ctypes.byref(bad))
    return out, bad.value


def gauss_legendre(p, q: int, nthreads: int = 1):
    """Tensor Gauss-Legendre integral over [0,1]^d of the untransformed integrand."""
    x, w = np.polynomial.legendre.leggauss(q)
    nodes = np.ascontiguousarray(0.5 * (x + 1.0))
    weights = np.ascontiguousarray(0.5 * w)
    mp = _Marshalled(p)
    out = np.zeros(2)
    lib().orc_gauss_legendre(ctypes.byref(mp.s), q, _ptr(nodes), _ptr(weights), max(1, int(nthreads)), _ptr(out))
    return out


def det_lu(a):
    """Determinant of a complex square matrix by LU with partial pivoting."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    d = a.shape[0]
    out = np.zeros(2)
    work = a.copy()
    lib().orc_det_lu_out(d, _ptr(work), _ptr(out))
    return complex(out[0], out[1])


def cv_g(d, R, K, F, a, x) -> float:
    """Control-variate surrogate g(x) = sum_r prod_i sum_k a_rik cos(F pi k x_i)."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    return float(lib().orc_cv_g(d, R, K, F, _ptr(a), _ptr(x)))


def cv_integral(d, R, K, a) -> float:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    return float(lib().orc_cv_integral(d, R, K, _ptr(a)))


def cv_loss_grad(d, R, K, F, x, h, a):
    """(loss, grad[R*d*K]) of the mean squared fit, FP64."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    h = np.ascontiguousarray(np.asarray(h, dtype=np.float64))
    grad = np.zeros(R * d * K)
    loss = lib().orc_cv_loss_grad(d, R, K, F, h.shape[0], _ptr(x), _ptr(h), _ptr(a), _ptr(grad))
    return float(loss), grad


def cv_loss_grad_bf16(d, R, K, F, x, h, a):
    """(loss, grad[R*d*K]) of the fit with BF16-rounded contraction operands, FP64 sums."""
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    h = np.ascontiguousarray(np.asarray(h, dtype=np.float64))
    grad = np.zeros(R * d * K)
    loss = lib().orc_cv_loss_grad_bf16(d, R, K, F, h.shape[0], _ptr(x), _ptr(h), _ptr(a), _ptr(grad))
    return float(loss), grad


def bf16(v: float) -> float:
    """v rounded to float, then to bfloat16 (nearest, ties to even)."""
    return float(lib().orc_bf16(float(v)))


def cbc_error(d: int, n: int, g, gamma) -> float:
    g = np.ascontiguousarray(np.asarray(g, dtype=np.uint64))
    gamma = np.ascontiguousarray(np.asarray(gamma, dtype=np.float64))
    return float(lib().orc_cbc_error(d, n, _ptr(g), _ptr(gamma)))


def cbc_candidate(n: int, p, z: int) -> float:
    """T(z) = sum_k p[k] B2({k z / n}) (Neumaier, k ascending)."""
    p = np.ascontiguousarray(np.asarray(p, dtype=np.float64))
    return float(lib().orc_cbc_candidate(n, _ptr(p), z))


def cbc_plain(d: int, n: int, gamma) -> np.ndarray:
    gamma = np.ascontiguousarray(np.asarray(gamma, dtype=np.float64))
    g = np.zeros(d, dtype=np.uint64)
    if lib().orc_cbc_plain(d, n, _ptr(gamma), _ptr(g)) != 0:
        raise ValueError("bad CBC arguments")
    return g

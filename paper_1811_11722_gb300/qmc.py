"""ctypes binding of libqmc_gb300.so (include/qmc.h), argument marshalling only.

Every function keeps the C name and forwards to the library; all arithmetic of
the rule runs in the CUDA library.  Loading fails loudly when the library has
not been built (``python -m paper_1811_11722_gb300.build``): there is no CPU
fallback.

Host inputs are numpy arrays.  Results may go to host memory (a qmc_result
returned here) or to device memory given as an integer address, e.g. a torch
CUDA tensor's ``data_ptr()``; streams are passed as integer handles, e.g.
``torch.cuda.current_stream().cuda_stream``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libqmc_gb300.so")

QMC_DMAX = 16
QMC_OK, QMC_EINVAL, QMC_ENOMEM, QMC_ECUDA = 0, -1, -2, -3
QMC_ENONFINITE, QMC_ETIMEOUT, QMC_EDEFORM, QMC_EUNSUPPORTED = -4, -5, -6, -7
QMC_TRANSFORM_NONE, QMC_TRANSFORM_KOROBOV, QMC_TRANSFORM_BAKER = 0, 1, 2
QMC_F_CONST, QMC_F_SEPARABLE_EXP, QMC_F_SECTOR, QMC_F_SECTOR_DEFORMED, QMC_F_TRIG = 0, 1, 2, 3, 4
QMC_FP64, QMC_FP32EVAL = 0, 1

STATUS_NAMES = {0: "QMC_OK", -1: "QMC_EINVAL", -2: "QMC_ENOMEM", -3: "QMC_ECUDA", -4: "QMC_ENONFINITE",
                -5: "QMC_ETIMEOUT", -6: "QMC_EDEFORM", -7: "QMC_EUNSUPPORTED"}
WARNINGS = (QMC_ENONFINITE, QMC_EDEFORM)


class QmcError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class qmc_transform(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("alpha", ctypes.c_int32)]


class qmc_poly(ctypes.Structure):
    _fields_ = [("nterms", ctypes.c_int32), ("coef", ctypes.c_void_p), ("expo", ctypes.c_void_p)]


class qmc_integrand(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("d", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("U", qmc_poly), ("F", qmc_poly), ("aU", ctypes.c_int32), ("aF", ctypes.c_int32),
                ("lam", ctypes.c_double), ("c", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("h", ctypes.c_void_p)]


class qmc_result(ctypes.Structure):
    _fields_ = [("mean", ctypes.c_double * 2), ("var", ctypes.c_double * 2), ("err", ctypes.c_double * 2),
                ("nonfinite", ctypes.c_uint64), ("deform_violations", ctypes.c_uint64),
                ("status", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {"mean": np.array(self.mean[:]), "var": np.array(self.var[:]), "err": np.array(self.err[:]),
                "nonfinite": int(self.nonfinite), "deform_violations": int(self.deform_violations),
                "status": int(self.status)}


class qmc_problem(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int32), ("m", ctypes.c_int32), ("n", ctypes.c_uint64), ("g", ctypes.c_void_p),
                ("shifts", ctypes.c_void_p), ("t", qmc_transform), ("f", ctypes.POINTER(qmc_integrand))]


class qmc_eps(ctypes.Structure):
    _fields_ = [("orders", ctypes.c_int32), ("reserved", ctypes.c_int32), ("bU", ctypes.c_double),
                ("bF", ctypes.c_double)]


class qmc_cv_config(ctypes.Structure):
    _fields_ = [("R", ctypes.c_int32), ("K", ctypes.c_int32), ("freq_step", ctypes.c_int32), ("steps", ctypes.c_int32),
                ("lr", ctypes.c_float), ("band", ctypes.c_int32), ("seed", ctypes.c_uint64)]


RESULT_BYTES = ctypes.sizeof(qmc_result)

_lib = None
_lock = threading.Lock()


def lib():
    """Load libqmc_gb300.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1811_11722_gb300.build` "
                                  "(the rule has no CPU fallback)")
            L = ctypes.CDLL(LIB_PATH)
            vp, i32, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_uint64
            P_int = ctypes.POINTER(qmc_integrand)
            L.qmc_make_lattice.argtypes = [i32, u64, vp, vp]
            L.qmc_integrate.argtypes = [i32, u64, i32, vp, vp, qmc_transform, P_int, vp, vp, vp]
            L.qmc_plan_create.argtypes = [i32, u64, i32, vp, vp, qmc_transform, P_int, ctypes.POINTER(vp)]
            L.qmc_plan_execute.argtypes = [vp, vp, vp, vp]
            L.qmc_plan_destroy.argtypes = [vp]
            L.qmc_plan_launches.argtypes = [vp, ctypes.POINTER(i32)]
            L.qmc_plan_record_events.argtypes = [vp, vp, vp]
            L.qmc_plan_tune.argtypes = [vp, vp, ctypes.POINTER(i32)]
            L.qmc_plan_describe.argtypes = [vp, ctypes.c_char_p, i32]
            L.qmc_combine_shifts.argtypes = [i32, vp, vp]
            L.qmc_measure_peaks.argtypes = [vp, vp]
            L.qmc_integrate_to_tolerance.argtypes = [i32, i32, vp, vp, i32, vp, qmc_transform, P_int,
                                                     ctypes.c_double, vp, ctypes.POINTER(i32), vp]
            L.qmc_integrate_batch.argtypes = [i32, vp, vp, vp, vp]
            L.qmc_integrate_batch_to_tolerance.argtypes = [i32, vp, i32, vp, vp, i32, ctypes.c_double, i32, vp, vp,
                                                           ctypes.POINTER(i32), vp]
            L.qmc_integrate_batch_extensible.argtypes = [i32, vp, i32, vp, i32, ctypes.c_double, i32, vp, vp,
                                                         ctypes.POINTER(i32), vp]
            L.qmc_batch_plan_create.argtypes = [i32, vp, ctypes.POINTER(vp)]
            L.qmc_batch_plan_create_persistent.argtypes = [i32, vp, ctypes.c_uint32, ctypes.POINTER(vp)]
            L.qmc_batch_plan_execute.argtypes = [vp, vp, vp, vp]
            L.qmc_batch_plan_destroy.argtypes = [vp]
            L.qmc_batch_plan_launches.argtypes = [vp, ctypes.POINTER(i32)]
            L.qmc_batch_plan_describe.argtypes = [vp, ctypes.c_char_p, i32]
            L.qmc_batch_plan_tune.argtypes = [vp, vp, vp, ctypes.POINTER(u64)]
            L.qmc_sample_points.argtypes = [i32, u64, i32, vp, vp, qmc_transform, P_int, i32, vp, vp, vp, vp, vp, vp]
            P_cfg = ctypes.POINTER(qmc_cv_config)
            L.qmc_cv_train.argtypes = [i32, u64, vp, vp, qmc_transform, P_int, P_cfg, vp, vp, vp]
            L.qmc_integrate_cv.argtypes = [i32, u64, i32, vp, vp, qmc_transform, P_int, P_cfg, vp, vp, vp, vp]
            L.qmc_cv_loss_grad.argtypes = [i32, P_cfg, i32, vp, vp, vp, vp, vp, vp]
            L.qmc_integrate_cv_to_tolerance.argtypes = [i32, i32, vp, vp, i32, vp, qmc_transform, P_int, P_cfg, vp,
                                                        ctypes.c_double, vp, ctypes.POINTER(i32),
                                                        ctypes.POINTER(i32), vp, vp]
            L.qmc_integrate_noalloc.argtypes = [i32, u64, i32, vp, vp, qmc_transform, P_int, vp, vp, vp]
            P_eps = ctypes.POINTER(qmc_eps)
            L.qmc_integrate_eps.argtypes = [i32, u64, i32, vp, vp, qmc_transform, P_int, P_eps, vp, vp, vp]
            L.qmc_eps_plan_create.argtypes = [i32, u64, i32, vp, vp, qmc_transform, P_int, P_eps,
                                              ctypes.POINTER(vp)]
            L.qmc_sample_points_eps.argtypes = [i32, u64, i32, vp, vp, qmc_transform, P_int, P_eps, i32, vp, vp,
                                                vp, vp]
            L.qmc_integrate_multi.argtypes = [i32, u64, i32, vp, vp, qmc_transform, i32, vp, vp, vp, vp]
            L.qmc_multi_plan_create.argtypes = [i32, u64, i32, vp, vp, qmc_transform, i32, vp, ctypes.POINTER(vp)]
            L.qmc_make_lattice_embedded.argtypes = [i32, i32, i32, vp, i32, u64, vp]
            L.qmc_integrate_extensible.argtypes = [i32, i32, i32, vp, i32, vp, qmc_transform, P_int, ctypes.c_double,
                                                   vp, vp, vp, vp]
            L.qmc_last_error.restype = ctypes.c_char_p
            L.qmc_version.restype = i32
            for name in ("qmc_make_lattice", "qmc_integrate", "qmc_plan_create", "qmc_plan_execute",
                         "qmc_plan_destroy", "qmc_plan_launches", "qmc_plan_record_events", "qmc_plan_tune", "qmc_plan_describe", "qmc_integrate_batch", "qmc_batch_plan_create",
                         "qmc_batch_plan_execute", "qmc_batch_plan_destroy", "qmc_batch_plan_launches",
                         "qmc_batch_plan_tune", "qmc_sample_points", "qmc_cv_train", "qmc_integrate_cv",
                         "qmc_cv_loss_grad", "qmc_integrate_noalloc", "qmc_combine_shifts", "qmc_measure_peaks",
                         "qmc_integrate_to_tolerance", "qmc_integrate_eps", "qmc_eps_plan_create",
                         "qmc_sample_points_eps", "qmc_integrate_multi", "qmc_multi_plan_create", "qmc_make_lattice_embedded",
                         "qmc_integrate_extensible", "qmc_batch_plan_create_persistent",
                         "qmc_integrate_cv_to_tolerance", "qmc_batch_plan_describe",
                         "qmc_integrate_batch_to_tolerance", "qmc_integrate_batch_extensible"):
                getattr(L, name).restype = i32
            _lib = L
    return _lib


def qmc_last_error() -> str:
    return lib().qmc_last_error().decode()


def qmc_version() -> int:
    return int(lib().qmc_version())


def _check(rc: int, allow_warnings: bool = False) -> int:
    if rc == QMC_OK or (allow_warnings and rc in WARNINGS):
        return rc
    raise QmcError(rc, qmc_last_error())


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _addr(x):
    """Device/host address: an int, a numpy array, or an object with data_ptr()."""
    if x is None:
        return None
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    return _ptr(x)


# ------------------------------------------------------------- descriptors --

class Integrand:
    """Owns the numpy arrays behind a qmc_integrand (keep it alive across calls)."""

    def __init__(self, kind: int, d: int, precision: int = QMC_FP64, U=None, F=None, aU: int = -2, aF: int = -1,
                 lam: float = 0.0, c=None, b=None, h=None):
        self._keep = []
        s = qmc_integrand()
        s.kind, s.d, s.precision = kind, d, precision
        s.aU, s.aF, s.lam = aU, aF, float(lam)

        def arr(x, dt):
            if x is None:
                return None
            a = np.ascontiguousarray(np.asarray(x, dtype=dt))
            self._keep.append(a)
            return a

        for name, poly in (("U", U), ("F", F)):
            if poly is not None:
                coef, expo = poly
                ca, ea = arr(coef, np.float64), arr(expo, np.uint8)
                setattr(s, name, qmc_poly(ca.shape[0], _ptr(ca), _ptr(ea)))
        s.c = _ptr(arr(c, np.float64))
        s.b = _ptr(arr(b, np.float64))
        s.h = _ptr(arr(h, np.int32))
        self.s = s

    @property
    def ref(self):
        return ctypes.byref(self.s)


def transform(kind: str, alpha: int = 0) -> qmc_transform:
    k = {"none": QMC_TRANSFORM_NONE, "korobov": QMC_TRANSFORM_KOROBOV, "baker": QMC_TRANSFORM_BAKER}[kind]
    return qmc_transform(k, alpha)


def integrand_from_problem(p, precision: str | None = None) -> Integrand:
    """Integrand descriptor from a paper_1811_11722_gb300.inputs.Problem."""
    prec = {"fp64": QMC_FP64, "fp32": QMC_FP32EVAL}[precision or p.precision]
    kind = {"const": QMC_F_CONST, "separable_exp": QMC_F_SEPARABLE_EXP, "sector": QMC_F_SECTOR,
            "sector_deformed": QMC_F_SECTOR_DEFORMED, "trig": QMC_F_TRIG}[p.kind]
    U = (p.U.coef, p.U.expo) if p.U is not None else None
    F = (p.F.coef, p.F.expo) if p.F is not None else None
    return Integrand(kind, p.d, prec, U, F, p.aU, p.aF, p.lam, p.c, p.b, p.h)


# --------------------------------------------------------------- functions --

def qmc_make_lattice(d: int, n: int, gamma) -> np.ndarray:
    gamma = np.ascontiguousarray(np.asarray(gamma, dtype=np.float64))
    g = np.zeros(d, dtype=np.uint64)
    _check(lib().qmc_make_lattice(d, n, _ptr(gamma), _ptr(g)))
    return g


def qmc_integrate(d, n, m, g, shifts, t: qmc_transform, f: Integrand, out=None, per_shift=None, stream=0,
                  want_per_shift=False):
    """Returns (qmc_result, per_shift ndarray or None) for host outputs; with a
    device `out` address the call is asynchronous and returns (None, None)."""
    g = np.ascontiguousarray(np.asarray(g, dtype=np.uint64))
    shifts = np.ascontiguousarray(np.asarray(shifts, dtype=np.float64))
    if out is None:
        res = qmc_result()
        ps = np.zeros(2 * m) if (want_per_shift and per_shift is None) else per_shift
        rc = lib().qmc_integrate(d, n, m, _ptr(g), _ptr(shifts), t, f.ref, ctypes.byref(res), _addr(ps),
                                 ctypes.c_void_p(stream))
        _check(rc, allow_warnings=True)
        return res, (ps.reshape(m, 2) if isinstance(ps, np.ndarray) else None)
    rc = lib().qmc_integrate(d, n, m, _ptr(g), _ptr(shifts), t, f.ref, _addr(out), _addr(per_shift),
                             ctypes.c_void_p(stream))
    _check(rc, allow_warnings=True)
    return None, None


class Plan:
    """qmc_plan_create / qmc_plan_execute / qmc_plan_destroy.  With `eps`
    (a qmc_eps) the plan comes from qmc_eps_plan_create and execute() returns
    one result per epsilon order."""

    def __init__(self, d, n, m, g, shifts, t: qmc_transform, f: Integrand, eps: qmc_eps | None = None):
        self.m = m
        self._f = f
        self.orders = 1 if eps is None else int(eps.orders)
        g = np.ascontiguousarray(np.asarray(g, dtype=np.uint64))
        shifts = np.ascontiguousarray(np.asarray(shifts, dtype=np.float64))
        h = ctypes.c_void_p()
        if eps is None:
            _check(lib().qmc_plan_create(d, n, m, _ptr(g), _ptr(shifts), t, f.ref, ctypes.byref(h)))
        else:
            _check(lib().qmc_eps_plan_create(d, n, m, _ptr(g), _ptr(shifts), t, f.ref, ctypes.byref(eps),
                                             ctypes.byref(h)))
        self.h = h

    def execute(self, out=None, per_shift=None, stream=0):
        if out is None:
            res = (qmc_result * self.orders)()
            rc = lib().qmc_plan_execute(self.h, res, _addr(per_shift), ctypes.c_void_p(stream))
            _check(rc, allow_warnings=True)
            return res[0] if self.orders == 1 else list(res)
        _check(lib().qmc_plan_execute(self.h, _addr(out), _addr(per_shift), ctypes.c_void_p(stream)),
               allow_warnings=True)
        return None

    def tune(self, stream=0) -> int:
        """qmc_plan_tune: returns the chosen shifts-per-launch."""
        v = ctypes.c_int32(0)
        _check(lib().qmc_plan_tune(self.h, ctypes.c_void_p(stream), ctypes.byref(v)))
        return int(v.value)

    def record_events(self, before_rule=None, after_rule=None):
        """cudaEvent_t handles (ints) recorded around the rule kernels of later executes."""
        _check(lib().qmc_plan_record_events(self.h, ctypes.c_void_p(before_rule or 0),
                                            ctypes.c_void_p(after_rule or 0)))

    def launches(self) -> int:
        v = ctypes.c_int32(0)
        _check(lib().qmc_plan_launches(self.h, ctypes.byref(v)))
        return int(v.value)

    def describe(self) -> dict:
        buf = ctypes.create_string_buffer(256)
        _check(lib().qmc_plan_describe(self.h, buf, 256))
        return dict(kv.split("=") for kv in buf.value.decode().split())

    def destroy(self):
        if self.h:
            lib().qmc_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def qmc_plan_create(d, n, m, g, shifts, t, f) -> Plan:
    return Plan(d, n, m, g, shifts, t, f)


def qmc_plan_execute(plan: Plan, out=None, per_shift=None, stream=0):
    return plan.execute(out, per_shift, stream)


def qmc_plan_destroy(plan: Plan):
    plan.destroy()


class _Batch:
    """Marshalled qmc_problem array (keeps every referenced array alive)."""

    def __init__(self, problems):
        """problems: list of (d, n, m, g, shifts, qmc_transform, Integrand)."""
        self.keep = []
        self.arr = (qmc_problem * len(problems))()
        self.total_m = 0
        for i, (d, n, m, g, shifts, t, f) in enumerate(problems):
            g = np.ascontiguousarray(np.asarray(g, dtype=np.uint64))
            sh = np.ascontiguousarray(np.asarray(shifts, dtype=np.float64))
            self.keep += [g, sh, f]
            self.arr[i] = qmc_problem(d, m, n, _ptr(g), _ptr(sh), t, ctypes.pointer(f.s))
            self.total_m += m
        self.count = len(problems)


def qmc_integrate_batch(problems, stream=0, want_per_shift=False):
    b = _Batch(problems)
    res = (qmc_result * b.count)()
    ps = np.zeros(2 * b.total_m) if want_per_shift else None
    rc = lib().qmc_integrate_batch(b.count, ctypes.cast(b.arr, ctypes.c_void_p), ctypes.cast(res, ctypes.c_void_p),
                                   _ptr(ps), ctypes.c_void_p(stream))
    _check(rc, allow_warnings=True)
    return list(res), ps


WALK_SUM, WALK_EACH, WALK_PERSISTENT, WALK_JUMP = 0, 1, 0x10, 0x20


def qmc_integrate_batch_to_tolerance(problems, ladder_n, ladder_g, rel_tol, criterion=WALK_SUM, stream=0):
    """Per-problem ladder walk, each pass one batched launch: problem i starts
    on its own lattice, then takes the ladder lattices (ladder_n[l],
    ladder_g[l, :d_i]) above its n.  Returns (results, level index per problem
    (-1: its own lattice), passes, reached: bool)."""
    b = _Batch(problems)
    ladder_n = np.ascontiguousarray(np.asarray(ladder_n, dtype=np.uint64))
    if len(ladder_n) == 0:  # no ladder: every problem is evaluated on its own lattice only
        ladder_g = np.zeros((0, 8), dtype=np.uint64)
    else:
        ladder_g = np.ascontiguousarray(np.asarray(ladder_g, dtype=np.uint64).reshape(len(ladder_n), -1))
    res = (qmc_result * b.count)()
    lv = np.zeros(b.count, dtype=np.int32)
    passes = ctypes.c_int32(0)
    rc = lib().qmc_integrate_batch_to_tolerance(b.count, ctypes.cast(b.arr, ctypes.c_void_p), len(ladder_n),
                                                _ptr(ladder_n), _ptr(ladder_g), ladder_g.shape[1],
                                                float(rel_tol), int(criterion), ctypes.cast(res, ctypes.c_void_p),
                                                _ptr(lv), ctypes.byref(passes), ctypes.c_void_p(stream))
    if rc != QMC_ETIMEOUT:
        _check(rc, allow_warnings=True)
    return list(res), lv, int(passes.value), rc != QMC_ETIMEOUT


def qmc_integrate_batch_extensible(problems, levels, g, rel_tol, criterion=WALK_SUM, stream=0):
    """Per-problem doubling walk on embedded base-2 lattices, each pass one
    batched launch: problem i starts with the rule of its n = 2^k points on
    g[:d_i] mod n (its own g is not read).  Returns (results, doublings per
    problem, passes, reached: bool)."""
    b = _Batch(problems)
    g = np.ascontiguousarray(np.asarray(g, dtype=np.uint64))
    res = (qmc_result * b.count)()
    lv = np.zeros(b.count, dtype=np.int32)
    passes = ctypes.c_int32(0)
    rc = lib().qmc_integrate_batch_extensible(b.count, ctypes.cast(b.arr, ctypes.c_void_p), int(levels), _ptr(g),
                                              len(g), float(rel_tol), int(criterion), ctypes.cast(res, ctypes.c_void_p),
                                              _ptr(lv), ctypes.byref(passes), ctypes.c_void_p(stream))
    if rc != QMC_ETIMEOUT:
        _check(rc, allow_warnings=True)
    return list(res), lv, int(passes.value), rc != QMC_ETIMEOUT


class BatchPlan:
    """qmc_batch_plan_create (a graph of per-problem kernels) or, with
    persistent=True, qmc_batch_plan_create_persistent (one persistent launch,
    `chunk` points per work item, 0 = the library default); _execute /
    _destroy."""

    def __init__(self, problems, persistent=False, chunk=0):
        self.b = _Batch(problems)
        h = ctypes.c_void_p()
        arr = ctypes.cast(self.b.arr, ctypes.c_void_p)
        if persistent:
            _check(lib().qmc_batch_plan_create_persistent(self.b.count, arr, int(chunk), ctypes.byref(h)))
        else:
            _check(lib().qmc_batch_plan_create(self.b.count, arr, ctypes.byref(h)))
        self.h = h

    def execute(self, out=None, per_shift=None, stream=0):
        if out is None:
            res = (qmc_result * self.b.count)()
            rc = lib().qmc_batch_plan_execute(self.h, ctypes.cast(res, ctypes.c_void_p), _addr(per_shift),
                                              ctypes.c_void_p(stream))
            _check(rc, allow_warnings=True)
            return list(res)
        _check(lib().qmc_batch_plan_execute(self.h, _addr(out), _addr(per_shift), ctypes.c_void_p(stream)),
               allow_warnings=True)
        return None

    def launches(self) -> int:
        v = ctypes.c_int32(0)
        _check(lib().qmc_batch_plan_launches(self.h, ctypes.byref(v)))
        return int(v.value)

    def describe(self) -> dict:
        buf = ctypes.create_string_buffer(256)
        _check(lib().qmc_batch_plan_describe(self.h, buf, 256))
        return dict(kv.split("=") for kv in buf.value.decode().split())

    def tune(self, stream=0) -> int:
        w = ctypes.c_uint64(0)
        _check(lib().qmc_batch_plan_tune(self.h, ctypes.cast(self.b.arr, ctypes.c_void_p), ctypes.c_void_p(stream),
                                         ctypes.byref(w)))
        return int(w.value)

    def destroy(self):
        if self.h:
            lib().qmc_batch_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def qmc_sample_points(d, n, m, g, shifts, t, f: Integrand, j, k, want_idx=True, want_coord=True, stream=0):
    """Returns (values[count, 2], idx[count, d] or None, coord[count, d] or None)."""
    g = np.ascontiguousarray(np.asarray(g, dtype=np.uint64))
    shifts = np.ascontiguousarray(np.asarray(shifts, dtype=np.float64))
    j = np.ascontiguousarray(np.asarray(j, dtype=np.uint64))
    k = np.ascontiguousarray(np.asarray(k, dtype=np.int32))
    cnt = j.shape[0]
    vals = np.zeros((cnt, 2))
    idx = np.zeros((cnt, d), dtype=np.uint64) if want_idx else None
    crd = np.zeros((cnt, d)) if want_coord else None
    _check(lib().qmc_sample_points(d, n, m, _ptr(g), _ptr(shifts), t, f.ref, cnt, _ptr(j), _ptr(k), _ptr(vals),
                                   _ptr(idx), _ptr(crd), ctypes.c_void_p(stream)))
    return vals, idx, crd


# --------------------------------------------------- embedded lattices --

def qmc_make_lattice_embedded(d: int, log2_nmin: int, log2_nmax: int, gamma, candidates: int = 1 << 30,
                              seed: int = 0) -> np.ndarray:
    gamma = np.ascontiguousarray(np.asarray(gamma, dtype=np.float64))
    g = np.zeros(d, dtype=np.uint64)
    _check(lib().qmc_make_lattice_embedded(d, log2_nmin, log2_nmax, _ptr(gamma), int(min(candidates, 2**31 - 1)),
                                           seed, _ptr(g)))
    return g


def qmc_integrate_extensible(d, log2_n0, levels, g, m, shifts, t, f: Integrand, rel_tol, stream=0):
    """Returns (qmc_result, level reached, per_shift[m, 2], tolerance met)."""
    g = np.ascontiguousarray(np.asarray(g, dtype=np.uint64))
    shifts = np.ascontiguousarray(np.asarray(shifts, dtype=np.float64))
    res = qmc_result()
    ps = np.zeros((m, 2))
    lvl = ctypes.c_int32(-1)
    rc = lib().qmc_integrate_extensible(d, log2_n0, levels, _ptr(g), m, _ptr(shifts), t, f.ref, float(rel_tol),
                                        ctypes.byref(res), _ptr(ps), ctypes.byref(lvl), ctypes.c_void_p(stream))
    if rc == QMC_ETIMEOUT:
        return res, int(lvl.value), ps, False
    _check(rc, allow_warnings=True)
    return res, int(lvl.value), ps, True


# ------------------------------------------------------- epsilon expansion --

def eps_spec(orders: int, bU: float = 1.0, bF: float = -1.0) -> qmc_eps:
    """Orders f_0..f_{orders-1} of U^(aU + bU eps) F^(aF + bF eps) (Eq. 7)."""
    return qmc_eps(int(orders), 0, float(bU), float(bF))


def qmc_integrate_eps(d, n, m, g, shifts, t, f: Integrand, eps: qmc_eps, want_per_shift=False, stream=0):
    """Returns (list of qmc_result, one per order; per_shift[orders, m, 2] or None)."""
    g = np.ascontiguousarray(np.asarray(g, dtype=np.uint64))
    shifts = np.ascontiguousarray(np.asarray(shifts, dtype=np.float64))
    res = (qmc_result * eps.orders)()
    ps = np.zeros((eps.orders, m, 2)) if want_per_shift else None
    rc = lib().qmc_integrate_eps(d, n, m, _ptr(g), _ptr(shifts), t, f.ref, ctypes.byref(eps), res, _ptr(ps),
                                 ctypes.c_void_p(stream))
    _check(rc, allow_warnings=True)
    return list(res), ps


def qmc_eps_plan_create(d, n, m, g, shifts, t, f: Integrand, eps: qmc_eps) -> Plan:
    return Plan(d, n, m, g, shifts, t, f, eps)


def qmc_sample_points_eps(d, n, m, g, shifts, t, f: Integrand, eps: qmc_eps, j, k, stream=0):
    """values[count, orders]: order o of the weighted value at (j[s], k[s])."""
    g = np.ascontiguousarray(np.asarray(g, dtype=np.uint64))
    shifts = np.ascontiguousarray(np.asarray(shifts, dtype=np.float64))
    j = np.ascontiguousarray(np.asarray(j, dtype=np.uint64))
    k = np.ascontiguousarray(np.asarray(k, dtype=np.int32))
    vals = np.zeros((j.shape[0], eps.orders))
    _check(lib().qmc_sample_points_eps(d, n, m, _ptr(g), _ptr(shifts), t, f.ref, ctypes.byref(eps), j.shape[0],
                                       _ptr(j), _ptr(k), _ptr(vals), ctypes.c_void_p(stream)))
    return vals


# ------------------------------------------- several integrands, one lattice --

def _integrand_array(fs):
    arr = (qmc_integrand * len(fs))()
    for s, f in enumerate(fs):
        arr[s] = f.s
    return arr


def qmc_integrate_multi(d, n, m, g, shifts, t, fs, want_per_shift=False, stream=0):
    """Integrands fs (list of Integrand) on one lattice.  Returns (results
    [len(fs) + 1], the last for their sum; per_shift[len(fs) + 1, m, 2] or None)."""
    g = np.ascontiguousarray(np.asarray(g, dtype=np.uint64))
    shifts = np.ascontiguousarray(np.asarray(shifts, dtype=np.float64))
    arr = _integrand_array(fs)
    res = (qmc_result * (len(fs) + 1))()
    ps = np.zeros((len(fs) + 1, m, 2)) if want_per_shift else None
    rc = lib().qmc_integrate_multi(d, n, m, _ptr(g), _ptr(shifts), t, len(fs), arr, res, _ptr(ps),
                                   ctypes.c_void_p(stream))
    _check(rc, allow_warnings=True)
    return list(res), ps


class MultiPlan(Plan):
    """qmc_multi_plan_create; execute() returns len(fs) + 1 results."""

    def __init__(self, d, n, m, g, shifts, t, fs):
        self.m = m
        self._fs = list(fs)
        self.orders = len(fs) + 1
        g = np.ascontiguousarray(np.asarray(g, dtype=np.uint64))
        shifts = np.ascontiguousarray(np.asarray(shifts, dtype=np.float64))
        arr = _integrand_array(fs)
        h = ctypes.c_void_p()
        _check(lib().qmc_multi_plan_create(d, n, m, _ptr(g), _ptr(shifts), t, len(fs), arr, ctypes.byref(h)))
        self.h = h


def qmc_multi_plan_create(d, n, m, g, shifts, t, fs) -> MultiPlan:
    return MultiPlan(d, n, m, g, shifts, t, fs)


# --------------------------------------------------------- control variate --

def qmc_cv_train(d, n_pilot, g_pilot, shift_pilot, t, f: Integrand, cfg: qmc_cv_config, stream=0):
    """Returns (a[R*d*K] float32 holding bfloat16 values, losses[2])."""
    g = np.ascontiguousarray(np.asarray(g_pilot, dtype=np.uint64))
    sh = np.ascontiguousarray(np.asarray(shift_pilot, dtype=np.float64))
    a = np.zeros(cfg.R * d * cfg.K, dtype=np.float32)
    losses = np.zeros(2)
    _check(lib().qmc_cv_train(d, n_pilot, _ptr(g), _ptr(sh), t, f.ref, ctypes.byref(cfg), _ptr(a), _ptr(losses),
                              ctypes.c_void_p(stream)))
    return a, losses


def qmc_integrate_cv(d, n, m, g, shifts, t, f: Integrand, cfg: qmc_cv_config, a, stream=0):
    """Returns (qmc_result with [0] = control variate, [1] = plain; per_shift[m, 2])."""
    g = np.ascontiguousarray(np.asarray(g, dtype=np.uint64))
    shifts = np.ascontiguousarray(np.asarray(shifts, dtype=np.float64))
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    res = qmc_result()
    ps = np.zeros(2 * m)
    rc = lib().qmc_integrate_cv(d, n, m, _ptr(g), _ptr(shifts), t, f.ref, ctypes.byref(cfg), _ptr(a),
                                ctypes.byref(res), _ptr(ps), ctypes.c_void_p(stream))
    _check(rc, allow_warnings=True)
    return res, ps.reshape(m, 2)


def qmc_cv_loss_grad(d, cfg: qmc_cv_config, x, h, a, stream=0):
    x = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    h = np.ascontiguousarray(np.asarray(h, dtype=np.float64))
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    loss = ctypes.c_double(0.0)
    grad = np.zeros(a.shape[0], dtype=np.float32)
    _check(lib().qmc_cv_loss_grad(d, ctypes.byref(cfg), h.shape[0], _ptr(x), _ptr(h), _ptr(a), ctypes.byref(loss),
                                  _ptr(grad), ctypes.c_void_p(stream)))
    return float(loss.value), grad


def qmc_integrate_noalloc(d, n, m, g, shifts, t: qmc_transform, f: Integrand, out=None, per_shift=None, stream=0):
    """qmc_integrate without device allocation (fixed per-device scratch array).
    Host result by default; with a device `out` address the call is asynchronous."""
    g = np.ascontiguousarray(np.asarray(g, dtype=np.uint64))
    shifts = np.ascontiguousarray(np.asarray(shifts, dtype=np.float64))
    if out is None:
        res = qmc_result()
        ps = np.zeros(2 * m) if per_shift is None else per_shift
        rc = lib().qmc_integrate_noalloc(d, n, m, _ptr(g), _ptr(shifts), t, f.ref, ctypes.byref(res), _addr(ps),
                                         ctypes.c_void_p(stream))
        _check(rc, allow_warnings=True)
        return res, (ps.reshape(m, 2) if isinstance(ps, np.ndarray) else None)
    rc = lib().qmc_integrate_noalloc(d, n, m, _ptr(g), _ptr(shifts), t, f.ref, _addr(out), _addr(per_shift),
                                     ctypes.c_void_p(stream))
    _check(rc, allow_warnings=True)
    return None, None


def qmc_combine_shifts(per_shift) -> qmc_result:
    """Eq. (3) over the rows (Q^(k) re, im) of per_shift[m, 2] (host computation)."""
    ps = np.ascontiguousarray(np.asarray(per_shift, dtype=np.float64).reshape(-1, 2))
    res = qmc_result()
    _check(lib().qmc_combine_shifts(ps.shape[0], _ptr(ps), ctypes.byref(res)))
    return res


def qmc_measure_peaks(stream=0) -> dict:
    """Measured FP32 / FP64 FMA and warp-level TF32 / BF16 MMA TFLOP/s of the current GPU."""
    out = np.zeros(4)
    _check(lib().qmc_measure_peaks(ctypes.c_void_p(stream), _ptr(out)))
    return {"fp32_tflops": float(out[0]), "fp64_tflops": float(out[1]), "mma_sync_tf32_tflops": float(out[2]),
            "mma_sync_bf16_tflops": float(out[3])}


def qmc_integrate_cv_to_tolerance(d, ns, gs, m, shifts, t, f: Integrand, cfg: qmc_cv_config, a, rel_tol, stream=0):
    """The control-variate ladder with its pilot judge.  Returns (qmc_result,
    level index, mode (1 control variate kept, 0 plain rule), judge dict,
    reached: bool)."""
    ns = np.ascontiguousarray(np.asarray(ns, dtype=np.uint64))
    gs = np.ascontiguousarray(np.asarray(gs, dtype=np.uint64).reshape(len(ns), d))
    shifts = np.ascontiguousarray(np.asarray(shifts, dtype=np.float64))
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    res = qmc_result()
    lvl, mode = ctypes.c_int32(-1), ctypes.c_int32(-1)
    judge = np.zeros(8)
    rc = lib().qmc_integrate_cv_to_tolerance(d, len(ns), _ptr(ns), _ptr(gs), m, _ptr(shifts), t, f.ref,
                                             ctypes.byref(cfg), _ptr(a), rel_tol, ctypes.byref(res),
                                             ctypes.byref(lvl), ctypes.byref(mode), _ptr(judge),
                                             ctypes.c_void_p(stream))
    if rc not in (QMC_OK, QMC_ETIMEOUT) and rc not in WARNINGS:
        _check(rc)
    j = {"rel_err_cv": float(judge[0]), "rel_err_plain": float(judge[1]), "pass_s_cv": float(judge[2]),
         "pass_s_plain": float(judge[3]), "rate_cv": float(judge[4]), "rate_plain": float(judge[5]),
         "predicted_s_cv": float(judge[6]), "predicted_s_plain": float(judge[7])}
    return res, int(lvl.value), int(mode.value), j, rc != QMC_ETIMEOUT


def qmc_integrate_to_tolerance(d, ns, gs, m, shifts, t, f: Integrand, rel_tol, stream=0):
    """Walk the lattices (ns[l], gs[l]) until err/|Qbar| <= rel_tol.
    Returns (qmc_result, level index, reached: bool)."""
    ns = np.ascontiguousarray(np.asarray(ns, dtype=np.uint64))
    gs = np.ascontiguousarray(np.asarray(gs, dtype=np.uint64).reshape(len(ns), d))
    shifts = np.ascontiguousarray(np.asarray(shifts, dtype=np.float64))
    res = qmc_result()
    lvl = ctypes.c_int32(-1)
    rc = lib().qmc_integrate_to_tolerance(d, len(ns), _ptr(ns), _ptr(gs), m, _ptr(shifts), t, f.ref, rel_tol,
                                          ctypes.byref(res), ctypes.byref(lvl), ctypes.c_void_p(stream))
    if rc not in (QMC_OK, QMC_ETIMEOUT) and rc not in WARNINGS:
        _check(rc)
    return res, int(lvl.value), rc != QMC_ETIMEOUT

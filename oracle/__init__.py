"""CPU FP64 oracle for restarted PDHG (arXiv 2312.14832, Section 2).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU-baseline leg, never by the solver package.  The arithmetic lives
in ``pdlp_oracle.c`` (plain loops, IEEE double, no FMA contraction); this module
compiles it with gcc on first use and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pdlp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

STATUS_OPTIMAL = 0
STATUS_ITER_LIMIT = 1


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared",
                                   "-fPIC", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int64), ("check_every", C.c_int32),
                ("scaling", C.c_int32), ("beta_suff", C.c_double), ("beta_nec", C.c_double),
                ("beta_art", C.c_double), ("step_scale", C.c_double), ("omega_theta", C.c_double),
                ("ruiz_iters", C.c_int32), ("power_iters", C.c_int32), ("eta", C.c_double),
                ("omega0", C.c_double), ("step_rule", C.c_int32), ("reject_cap", C.c_int32)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("which", C.c_int32), ("iters", C.c_int64),
                ("restarts", C.c_int64), ("primal_obj", C.c_double), ("dual_obj", C.c_double),
                ("rel_primal", C.c_double), ("rel_dual", C.c_double), ("rel_gap", C.c_double),
                ("kkt_omega", C.c_double), ("omega", C.c_double), ("eta", C.c_double),
                ("accepted", C.c_int64), ("checks", C.c_int64)]


class CheckRecord(C.Structure):
    _fields_ = [("k", C.c_int64), ("t", C.c_int64), ("restart", C.c_int32), ("candidate", C.c_int32),
                ("omega", C.c_double), ("kkt_cur", C.c_double), ("kkt_avg", C.c_double),
                ("kkt_anchor", C.c_double), ("rel_primal", C.c_double), ("rel_dual", C.c_double),
                ("rel_gap", C.c_double)]


class KKT(C.Structure):
    _fields_ = [("pres2", C.c_double), ("dres2", C.c_double), ("pobj", C.c_double),
                ("dobj", C.c_double), ("gap", C.c_double)]


_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_vp = C.c_void_p


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        L.orc_spmv.argtypes = [C.c_int64, _i64p, _i32p, _dp, _dp, _dp]
        L.orc_spmv_t.argtypes = [C.c_int64, C.c_int64, _i64p, _i32p, _dp, _dp, _dp]
        L.orc_proj_lambda.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_proj_lambda.restype = C.c_double
        L.orc_kkt_parts.argtypes = [C.c_int64, C.c_int64, C.c_int64, _i64p, _i32p, _dp, _dp, _dp,
                                    _dp, _dp, _dp, _dp]
        L.orc_kkt_parts.restype = KKT
        L.orc_kkt_omega.argtypes = [KKT, C.c_double]
        L.orc_kkt_omega.restype = C.c_double
        L.orc_restart_decision.argtypes = [C.c_double, C.c_double, C.c_double, C.c_int64, C.c_int64,
                                           C.c_double, C.c_double, C.c_double]
        L.orc_restart_decision.restype = C.c_int
        L.orc_restart_candidate.argtypes = [C.c_double, C.c_double]
        L.orc_restart_candidate.restype = C.c_int
        L.orc_scale.argtypes = [C.c_int64, C.c_int64, _i64p, _i32p, _dp, C.c_int32, C.c_int32, _dp, _dp]
        L.orc_power_norm.argtypes = [C.c_int64, C.c_int64, _i64p, _i32p, _dp, C.c_int32]
        L.orc_power_norm.restype = C.c_double
        L.orc_pdhg_step.argtypes = [C.c_int64, C.c_int64, C.c_int64, _i64p, _i32p, _dp, _dp, _dp,
                                    _dp, _dp, C.c_double, C.c_double, _dp, _dp]
        L.orc_transpose.argtypes = [C.c_int64, C.c_int64, _i64p, _i32p, _dp, _i64p, _i32p, _dp]
        L.orc_pdhg_step_par.argtypes = [C.c_int64, C.c_int64, C.c_int64, _i64p, _i32p, _dp, _i64p, _i32p, _dp,
                                        _dp, _dp, _dp, _dp, C.c_double, C.c_double, _dp, _dp, C.c_int32]
        L.orc_solve.argtypes = [C.c_int64, C.c_int64, C.c_int64, _i64p, _i32p, _dp, _dp, _dp, _dp,
                                _dp, C.POINTER(Params), _vp, _vp, C.POINTER(Result), _vp, _vp, _vp,
                                _vp, _vp, _vp, _vp, C.c_int64, _vp, C.c_int64]
        L.orc_solve.restype = C.c_int
        _lib = L
    return _lib


def default_params(**kw) -> Params:
    p = Params(tol=1e-4, max_iter=100_000_000, check_every=64, scaling=0, beta_suff=0.2,
               beta_nec=0.8, beta_art=0.36, step_scale=0.9, omega_theta=0.5, ruiz_iters=10,
               power_iters=100, eta=0.0, omega0=0.0, reject_cap=64)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _csr(lp):
    return (np.ascontiguousarray(lp["row_ptr"], dtype=np.int64),
            np.ascontiguousarray(lp["col_idx"], dtype=np.int32),
            _f64(lp["val"]))


def spmv(lp, x):
    rp, ci, v = _csr(lp)
    y = np.zeros(max(lp["m"], 1))
    lib().orc_spmv(lp["m"], rp, ci, v, _f64(x) if lp["n"] else np.zeros(1), y)
    return y[: lp["m"]]


def spmv_t(lp, y):
    rp, ci, v = _csr(lp)
    g = np.zeros(max(lp["n"], 1))
    lib().orc_spmv_t(lp["m"], lp["n"], rp, ci, v, _f64(y) if lp["m"] else np.zeros(1), g)
    return g[: lp["n"]]


def proj_lambda(d, l, u):
    return lib().orc_proj_lambda(float(d), float(l), float(u))


def _pad(a):
    a = _f64(a)
    return a if a.shape[0] else np.zeros(1)


def kkt_parts(lp, x, y):
    """(pres2, dres2, pobj, dobj, gap) of (x, y) for the LP as given (no scaling)."""
    rp, ci, v = _csr(lp)
    r = lib().orc_kkt_parts(lp["m"], lp["n"], lp["m1"], rp, ci, v, _pad(lp["c"]), _pad(lp["q"]),
                            _pad(lp["l"]), _pad(lp["u"]), _pad(x), _pad(y))
    return dict(pres2=r.pres2, dres2=r.dres2, pobj=r.pobj, dobj=r.dobj, gap=r.gap)


def kkt_omega(parts, omega):
    return lib().orc_kkt_omega(KKT(**parts), float(omega))


def relative_errors(lp, x, y):
    """The three relative termination ratios of Section 2 on the LP as given."""
    p = kkt_parts(lp, x, y)
    qn = float(np.linalg.norm(lp["q"]))
    cn = float(np.linalg.norm(lp["c"]))
    return (np.sqrt(p["pres2"]) / (1 + qn), np.sqrt(p["dres2"]) / (1 + cn),
            abs(p["gap"]) / (1 + abs(p["dobj"]) + abs(p["pobj"])))


def restart_decision(kkt_c, kkt_anchor, kkt_prev_c, t, k, beta_suff=0.2, beta_nec=0.8, beta_art=0.36):
    return lib().orc_restart_decision(kkt_c, kkt_anchor, kkt_prev_c, t, k, beta_suff, beta_nec, beta_art)


def restart_candidate(kkt_cur, kkt_avg):
    """1 when the restart candidate is the average, 0 for the current iterate."""
    return lib().orc_restart_candidate(float(kkt_cur), float(kkt_avg))


def scale(lp, ruiz_iters=10, pock_chambolle=True):
    """Returns (scaled values, Dr, Dc)."""
    rp, ci, v = _csr(lp)
    v = v.copy() if v.shape[0] else np.zeros(1)
    Dr = np.zeros(max(lp["m"], 1))
    Dc = np.zeros(max(lp["n"], 1))
    lib().orc_scale(lp["m"], lp["n"], rp, ci, v, ruiz_iters, int(pock_chambolle), Dr, Dc)
    return v[: lp["val"].shape[0]], Dr[: lp["m"]], Dc[: lp["n"]]


def power_norm(lp, iters=100, val=None):
    rp, ci, v = _csr(lp)
    if val is not None:
        v = _f64(val)
    return lib().orc_power_norm(lp["m"], lp["n"], rp, ci, v if v.shape[0] else np.zeros(1), iters)


def pdhg_step(lp, x, y, eta, omega):
    """One PDHG step (primal update then dual update with extrapolation), unscaled LP."""
    rp, ci, v = _csr(lp)
    x = _f64(x).copy()
    y = _f64(y).copy()
    xx, yy = _pad(x).copy(), _pad(y).copy()
    lib().orc_pdhg_step(lp["m"], lp["n"], lp["m1"], rp, ci, v if v.shape[0] else np.zeros(1),
                        _pad(lp["c"]), _pad(lp["q"]), _pad(lp["l"]), _pad(lp["u"]), float(eta),
                        float(omega), xx, yy)
    return xx[: lp["n"]], yy[: lp["m"]]


class ThreadedStep:
    """orc_pdhg_step on several host threads (the CPU baseline's all-core timing): K' is
    built once, then step(x, y) updates the point in place, bit-identical to pdhg_step."""

    def __init__(self, lp, threads):
        self.lp = lp
        self.threads = int(threads)
        self.rp, self.ci, self.v = _csr(lp)
        n, m = lp["n"], lp["m"]
        nnz = self.v.shape[0]
        self.tp = np.zeros(n + 1, dtype=np.int64)
        self.tc = np.zeros(max(nnz, 1), dtype=np.int32)
        self.tv = np.zeros(max(nnz, 1))
        lib().orc_transpose(m, n, self.rp, self.ci, self.v if nnz else np.zeros(1), self.tp, self.tc, self.tv)
        self.c, self.q, self.l, self.u = _pad(lp["c"]), _pad(lp["q"]), _pad(lp["l"]), _pad(lp["u"])

    def step(self, x, y, eta, omega):
        lp = self.lp
        lib().orc_pdhg_step_par(lp["m"], lp["n"], lp["m1"], self.rp, self.ci,
                                self.v if self.v.shape[0] else np.zeros(1), self.tp, self.tc, self.tv,
                                self.c, self.q, self.l, self.u, float(eta), float(omega), x, y, self.threads)


def solve(lp, params: Params | None = None, x0=None, y0=None, restart_cap=1 << 16, log_cap=0, **kw):
    """Restarted PDHG.  Returns a dict with the result fields, x/y (returned point),
    x_cur/y_cur, x_avg/y_avg (unscaled), the list of restart iterations and, when
    log_cap > 0, the first log_cap per-check records as dicts ("log")."""
    p = params or default_params(**kw)
    if params is not None:
        for k, v in kw.items():
            setattr(p, k, v)
    m, n = lp["m"], lp["n"]
    rp, ci, v = _csr(lp)
    bufs = {k: np.zeros(max(sz, 1)) for k, sz in
            (("x", n), ("y", m), ("x_cur", n), ("y_cur", m), ("x_avg", n), ("y_avg", m))}
    rs = np.zeros(restart_cap, dtype=np.int64)
    logbuf = (CheckRecord * max(log_cap, 1))()
    R = Result()
    x0p = _f64(x0).ctypes.data if x0 is not None else None
    y0p = _f64(y0).ctypes.data if y0 is not None else None
    keep = (None if x0 is None else _f64(x0), None if y0 is None else _f64(y0))
    if x0 is not None:
        x0p = keep[0].ctypes.data
    if y0 is not None:
        y0p = keep[1].ctypes.data
    rc = lib().orc_solve(m, n, lp["m1"], rp, ci, v if v.shape[0] else np.zeros(1), _pad(lp["c"]),
                         _pad(lp["q"]), _pad(lp["l"]), _pad(lp["u"]), C.byref(p), x0p, y0p,
                         C.byref(R), bufs["x"].ctypes.data, bufs["y"].ctypes.data,
                         bufs["x_cur"].ctypes.data, bufs["y_cur"].ctypes.data,
                         bufs["x_avg"].ctypes.data, bufs["y_avg"].ctypes.data, rs.ctypes.data,
                         restart_cap, C.addressof(logbuf) if log_cap > 0 else None, log_cap)
    if rc != 0:
        raise ValueError("oracle rejected the input")
    out = {f: getattr(R, f) for f, _ in Result._fields_}
    for k in ("x", "x_cur", "x_avg"):
        out[k] = bufs[k][:n]
    for k in ("y", "y_cur", "y_avg"):
        out[k] = bufs[k][:m]
    out["restart_iters"] = rs[: min(R.restarts, restart_cap)].copy()
    if log_cap > 0:
        out["log"] = [{f: getattr(r, f) for f, _ in CheckRecord._fields_}
                      for r in logbuf[: min(R.checks, log_cap)]]
    return out

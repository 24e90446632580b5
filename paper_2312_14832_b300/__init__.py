"""B300-native restarted PDHG for linear programming (arXiv 2312.14832, Section 2).

The solver is the native library ``libpdlp_b300.so`` (C ABI in include/pdlp.h, CUDA
kernels for sm_103a).  This module only marshals arguments: numpy arrays are passed
as host pointers, CUDA torch tensors as device pointers.  There is no CPU path: if
the library or a GPU is missing, the calls raise.

    lp = dict(m=..., n=..., m1=..., row_ptr=..., col_idx=..., val=..., c=..., q=..., l=..., u=...)
    with Solver.from_lp(lp, scaling=1) as s:
        r = s.solve(tol=1e-4)          # dict with status, iters, objectives, x, y, ...
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import FP64, ITER_LIMIT, MIXED, NUMERICAL, OPTIMAL, TIME_LIMIT  # noqa: F401

__all__ = ["Solver", "BatchSolver", "MLP", "SolverError", "default_params", "OPTIMAL", "ITER_LIMIT", "TIME_LIMIT",
           "NUMERICAL", "FP64", "MIXED"]


class SolverError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pdlp error {code}: {msg}")
        self.code = code


def default_params(**kw) -> _lib.Params:
    p = _lib.Params()
    _lib.load().pdlp_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(f"unknown parameter {k}")
        setattr(p, k, v)
    return p


def _info_dict(i) -> dict:
    out = {}
    for f, _ in _lib.Info._fields_:
        v = getattr(i, f)
        out[f] = list(v) if isinstance(v, C.Array) else v
    return out


def _is_torch_cuda(a) -> bool:
    return hasattr(a, "is_cuda") and bool(a.is_cuda)


class _Arg:
    """Keeps a contiguous array alive and exposes its address."""

    def __init__(self, a, dtype, device):
        if device:
            import torch
            tdt = {np.float64: torch.float64, np.int64: torch.int64, np.int32: torch.int32}[dtype]
            self.obj = a.to(dtype=tdt).contiguous()
            self.ptr = self.obj.data_ptr() if self.obj.numel() else None
        else:
            self.obj = np.ascontiguousarray(a, dtype=dtype)
            self.ptr = self.obj.ctypes.data if self.obj.size else None


class Solver:
    def __init__(self, m, n, m1, row_ptr, col_idx, val, c, q, l, u, **params):
        self._lib = _lib.load()
        self._h = C.c_void_p()
        self.m, self.n, self.m1 = int(m), int(n), int(m1)
        self.device = _is_torch_cuda(c)
        p = default_params(**params)
        p.inputs_on_device = 1 if self.device else 0
        if self.device and not p.stream:
            import torch
            p.stream = torch.cuda.current_stream().cuda_stream
        self.params = p
        args = [_Arg(row_ptr, np.int64, self.device), _Arg(col_idx, np.int32, self.device),
                _Arg(val, np.float64, self.device), _Arg(c, np.float64, self.device),
                _Arg(q, np.float64, self.device), _Arg(l, np.float64, self.device),
                _Arg(u, np.float64, self.device)]
        rc = self._lib.pdlp_setup(C.byref(self._h), self.m, self.n, self.m1,
                                  *[a.ptr for a in args], C.byref(p))
        if rc != 0:
            raise SolverError(rc, self._lib.pdlp_last_error(None).decode())

    @classmethod
    def from_lp(cls, lp, **params):
        return cls(lp["m"], lp["n"], lp["m1"], lp["row_ptr"], lp["col_idx"], lp["val"], lp["c"],
                   lp["q"], lp["l"], lp["u"], **params)

    # ------------------------------------------------------------------ helpers
    def _check(self, rc):
        if rc < 0:
            raise SolverError(rc, self._lib.pdlp_last_error(self._h).decode())
        return rc

    def _out(self, size):
        if self.device:
            import torch
            return torch.empty(max(size, 0), dtype=torch.float64, device="cuda")
        return np.empty(max(size, 0), dtype=np.float64)

    @staticmethod
    def _ptr(a):
        if a is None:
            return None
        if hasattr(a, "data_ptr"):
            return a.data_ptr() if a.numel() else None
        return a.ctypes.data if a.size else None

    # ------------------------------------------------------------------ API
    def solve(self, x0=None, y0=None, omega0=0.0, want_point=True, **overrides) -> dict:
        p = _lib.Params()
        C.memmove(C.byref(p), C.byref(self.params), C.sizeof(p))
        for k, v in overrides.items():
            if not hasattr(p, k):
                raise KeyError(f"unknown parameter {k}")
            setattr(p, k, v)
        xa = _Arg(x0, np.float64, self.device) if x0 is not None else None
        ya = _Arg(y0, np.float64, self.device) if y0 is not None else None
        x = self._out(self.n) if want_point else None
        y = self._out(self.m) if want_point else None
        r = _lib.Result()
        self._check(self._lib.pdlp_solve(self._h, C.byref(p), xa.ptr if xa else None,
                                         ya.ptr if ya else None, float(omega0), C.byref(r),
                                         self._ptr(x), self._ptr(y) if y is not None and self.m else None))
        out = {f: getattr(r, f) for f, _ in _lib.Result._fields_}
        out["x"], out["y"] = x, y
        return out

    def get_state(self) -> bytes:
        """The state of the last solve (pdlp_get_state): opaque bytes for resume()."""
        size = self._lib.pdlp_state_size(self._h)
        self._check(size)
        buf = C.create_string_buffer(int(size))
        self._check(self._lib.pdlp_get_state(self._h, buf, int(size)))
        return buf.raw

    def resume(self, state=None, want_point=True, **overrides) -> dict:
        """Continues the last solve of this handle, or the one saved in `state`
        (pdlp_solve_resume), until max_iter iterations in total or termination."""
        p = _lib.Params()
        C.memmove(C.byref(p), C.byref(self.params), C.sizeof(p))
        for k, v in overrides.items():
            if not hasattr(p, k):
                raise KeyError(f"unknown parameter {k}")
            setattr(p, k, v)
        buf = C.create_string_buffer(bytes(state), len(state)) if state is not None else None
        x = self._out(self.n) if want_point else None
        y = self._out(self.m) if want_point else None
        r = _lib.Result()
        self._check(self._lib.pdlp_solve_resume(self._h, C.byref(p), buf, len(state) if state is not None else 0,
                                                C.byref(r), self._ptr(x),
                                                self._ptr(y) if y is not None and self.m else None))
        out = {f: getattr(r, f) for f, _ in _lib.Result._fields_}
        out["x"], out["y"] = x, y
        return out

    def iterate(self, which=0):
        """which: 0 current iterate, 1 average of the inner loop, 2 restart anchor."""
        x, y = self._out(self.n), self._out(self.m)
        self._check(self._lib.pdlp_get_iterate(self._h, int(which), self._ptr(x),
                                               self._ptr(y) if self.m else None))
        return x, y

    def restarts(self):
        cnt = self._check(self._lib.pdlp_get_restarts(self._h, None, 0))
        buf = np.zeros(max(cnt, 1), dtype=np.int64)
        self._check(self._lib.pdlp_get_restarts(self._h, buf.ctypes.data, cnt))
        return buf[:cnt]

    def log(self):
        cnt = self._check(self._lib.pdlp_get_log(self._h, None, 0))
        recs = (_lib.CheckRecord * max(cnt, 1))()
        got = min(cnt, self.params.log_capacity)
        self._check(self._lib.pdlp_get_log(self._h, recs, got))
        return [{f: getattr(recs[i], f) for f, _ in _lib.CheckRecord._fields_} for i in range(got)]

    def spmv(self, v, transpose=False):
        """K v (transpose=False, v of length n) or K' v, through the device kernels."""
        a = _Arg(v, np.float64, self.device)
        out = self._out(self.n if transpose else self.m)
        if out.shape[0] == 0:
            return out
        self._check(self._lib.pdlp_spmv(self._h, 1 if transpose else 0, a.ptr, self._ptr(out)))
        return out

    def bound_duals(self, y):
        """lambda = proj_Lambda(c - K'y) on the original problem (the solver returns x, y)."""
        a = _Arg(y, np.float64, self.device) if self.m else None
        out = self._out(self.n)
        self._check(self._lib.pdlp_bound_duals(self._h, a.ptr if a else None, self._ptr(out)))
        return out

    def info(self) -> dict:
        i = _lib.Info()
        self._check(self._lib.pdlp_get_info(self._h, C.byref(i)))
        return _info_dict(i)

    def time_iterations(self, iters):
        a, b = C.c_double(), C.c_double()
        self._check(self._lib.pdlp_time_iterations(self._h, int(iters), C.byref(a), C.byref(b)))
        return a.value, b.value

    def close(self):
        if self._h:
            self._lib.pdlp_free(self._h)
            self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSolver:
    """Many independent LPs solved by one persistent kernel (pdlp_batch_setup/solve).

        with BatchSolver.from_lps([lp0, lp1, ...], scaling=1) as b:
            results = b.solve(tol=1e-4)     # one dict per LP, with x and y
    """

    def __init__(self, lps, **params):
        self._lib = _lib.load()
        self._h = C.c_void_p()
        self.count = len(lps)
        if self.count == 0:
            raise ValueError("empty batch")
        self.m = np.array([lp["m"] for lp in lps], dtype=np.int64)
        self.n = np.array([lp["n"] for lp in lps], dtype=np.int64)
        self.m1 = np.array([lp["m1"] for lp in lps], dtype=np.int64)
        cat = lambda key, dt: np.ascontiguousarray(np.concatenate([np.asarray(lp[key], dtype=dt) for lp in lps]))
        self._arrays = [cat("row_ptr", np.int64), cat("col_idx", np.int32), cat("val", np.float64),
                        cat("c", np.float64), cat("q", np.float64), cat("l", np.float64), cat("u", np.float64)]
        p = default_params(**params)
        p.inputs_on_device = 0
        self.params = p
        ptr = lambda a: a.ctypes.data if a.size else None
        rc = self._lib.pdlp_batch_setup(C.byref(self._h), self.count, self.m.ctypes.data, self.n.ctypes.data,
                                        self.m1.ctypes.data, *[ptr(a) for a in self._arrays], C.byref(p))
        if rc != 0:
            raise SolverError(rc, self._lib.pdlp_last_error(None).decode())
        self._arrays = None

    @classmethod
    def from_lps(cls, lps, **params):
        return cls(lps, **params)

    def solve(self, want_points=True, x0=None, y0=None, omega0=None, **overrides):
        """x0, y0: warm starts back to back (sum n, sum m) or per-LP lists; omega0: per LP."""
        p = _lib.Params()
        C.memmove(C.byref(p), C.byref(self.params), C.sizeof(p))
        for k, v in overrides.items():
            if not hasattr(p, k):
                raise KeyError(f"unknown parameter {k}")
            setattr(p, k, v)
        res = (_lib.Result * self.count)()
        x = np.empty(int(self.n.sum())) if want_points else None
        y = np.empty(int(self.m.sum())) if want_points else None
        cat = lambda v: None if v is None else np.ascontiguousarray(
            np.concatenate(v) if isinstance(v, (list, tuple)) else v, dtype=np.float64)
        x0a, y0a, w0a = cat(x0), cat(y0), (None if omega0 is None else np.ascontiguousarray(omega0, np.float64))
        if x0a is not None and x0a.shape[0] != int(self.n.sum()):
            raise ValueError("x0 must have sum(n) entries")
        if y0a is not None and y0a.shape[0] != int(self.m.sum()):
            raise ValueError("y0 must have sum(m) entries")
        if w0a is not None and w0a.shape[0] != self.count:
            raise ValueError("omega0 must have one entry per LP")
        ptr = lambda a: None if a is None or a.size == 0 else a.ctypes.data
        rc = self._lib.pdlp_batch_solve(self._h, C.byref(p), ptr(x0a), ptr(y0a), ptr(w0a), res,
                                        x.ctypes.data if want_points else None,
                                        y.ctypes.data if (want_points and y.size) else None)
        if rc < 0:
            raise SolverError(rc, self._lib.pdlp_last_error(self._h).decode())
        out = []
        xo = np.concatenate([[0], np.cumsum(self.n)])
        yo = np.concatenate([[0], np.cumsum(self.m)])
        for b in range(self.count):
            d = {f: getattr(res[b], f) for f, _ in _lib.Result._fields_}
            if want_points:
                d["x"] = x[xo[b]:xo[b + 1]].copy()
                d["y"] = y[yo[b]:yo[b + 1]].copy()
            out.append(d)
        return out

    def restarts(self, lp):
        """Iteration counts at which LP `lp` restarted in the last solve (the first 256)."""
        cnt = self._lib.pdlp_batch_get_restarts(self._h, int(lp), None, 0)
        if cnt < 0:
            raise SolverError(cnt, self._lib.pdlp_last_error(self._h).decode())
        buf = np.zeros(max(cnt, 1), dtype=np.int64)
        got = self._lib.pdlp_batch_get_restarts(self._h, int(lp), buf.ctypes.data, cnt)
        if got < 0:
            raise SolverError(got, self._lib.pdlp_last_error(self._h).decode())
        return buf[: min(cnt, 256)]

    def info(self) -> dict:
        """Layout sizes, the team size and resident mode of the last solve, and what the
        online autotuner timed (batch_tuned candidates: tune_team, tune_resident, tune_gbs)."""
        i = _lib.Info()
        rc = self._lib.pdlp_get_info(self._h, C.byref(i))
        if rc < 0:
            raise SolverError(rc, self._lib.pdlp_last_error(self._h).decode())
        return _info_dict(i)

    def spmv(self, v, transpose=False):
        """Block-diagonal K v (or K' v) of the whole batch."""
        a = np.ascontiguousarray(v, dtype=np.float64)
        out = np.empty(int(self.n.sum() if transpose else self.m.sum()))
        if out.size:
            rc = self._lib.pdlp_spmv(self._h, 1 if transpose else 0, a.ctypes.data, out.ctypes.data)
            if rc < 0:
                raise SolverError(rc, self._lib.pdlp_last_error(self._h).decode())
        return out

    def close(self):
        if self._h:
            self._lib.pdlp_free(self._h)
            self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MLP:
    """The warm-start network (pdlp_mlp_*): 3 linear layers with ReLU, BF16 tensor-core
    products, FP32 masters, AdamW.  Parameters are numpy float32 arrays
    W1 [hidden x n_in], b1, W2 [hidden x hidden], b2, W3 [n_out x hidden], b3."""

    def __init__(self, n_in, hidden, n_out, max_batch):
        self._lib = _lib.load()
        self._h = C.c_void_p()
        self.n_in, self.hidden, self.n_out, self.max_batch = n_in, hidden, n_out, max_batch
        rc = self._lib.pdlp_mlp_create(C.byref(self._h), n_in, hidden, n_out, max_batch)
        if rc != 0:
            raise SolverError(rc, self._lib.pdlp_last_error(None).decode())

    def _check(self, rc):
        if rc < 0:
            raise SolverError(rc, self._lib.pdlp_mlp_last_error(self._h).decode())

    def shapes(self):
        return [(self.hidden, self.n_in), (self.hidden,), (self.hidden, self.hidden), (self.hidden,),
                (self.n_out, self.hidden), (self.n_out,)]

    def set_params(self, params):
        arrs = [np.ascontiguousarray(p, dtype=np.float32) for p in params]
        for a, shp in zip(arrs, self.shapes()):
            if a.shape != shp:
                raise ValueError(f"parameter shape {a.shape} != {shp}")
        self._check(self._lib.pdlp_mlp_set_params(self._h, *[a.ctypes.data for a in arrs]))

    def get_params(self):
        arrs = [np.empty(shp, dtype=np.float32) for shp in self.shapes()]
        self._check(self._lib.pdlp_mlp_get_params(self._h, *[a.ctypes.data for a in arrs]))
        return arrs

    def load_data(self, X, T=None):
        self._X = np.ascontiguousarray(X, dtype=np.float32)
        self._T = None if T is None else np.ascontiguousarray(T, dtype=np.float32)
        self._check(self._lib.pdlp_mlp_load_data(self._h, self._X.shape[0], self._X.ctypes.data,
                                                 None if self._T is None else self._T.ctypes.data))
        self.count = self._X.shape[0]

    def forward(self, idx):
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        Y = np.empty((idx.shape[0], self.n_out), dtype=np.float32)
        for s in range(0, idx.shape[0], self.max_batch):
            part = np.ascontiguousarray(idx[s:s + self.max_batch])
            out = np.empty((part.shape[0], self.n_out), dtype=np.float32)
            self._check(self._lib.pdlp_mlp_forward(self._h, part.shape[0], part.ctypes.data, out.ctypes.data))
            Y[s:s + part.shape[0]] = out
        return Y

    def gradients(self, idx):
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        grads = [np.empty(shp, dtype=np.float32) for shp in self.shapes()]
        loss = C.c_double()
        self._check(self._lib.pdlp_mlp_gradients(self._h, idx.shape[0], idx.ctypes.data, C.byref(loss),
                                                 *[g.ctypes.data for g in grads]))
        return loss.value, grads

    def train(self, epochs, batch, lr, weight_decay=0.0, seed=0):
        losses = np.zeros(epochs)
        ms = C.c_double()
        self._check(self._lib.pdlp_mlp_train(self._h, epochs, batch, lr, weight_decay, seed, losses.ctypes.data,
                                             C.byref(ms)))
        return losses, ms.value

    def close(self):
        if self._h:
            self._lib.pdlp_mlp_free(self._h)
            self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

"""Learned warm start for a family of LPs (an extension of this library; the paper has no
learned component).

An MLP (``MLP``: three linear layers, ReLU, BF16 tcgen05 products, AdamW on the device)
maps the parameters of an LP of the family (for the transportation family: supplies
and demands) to a starting point x0, y0 and an initial primal weight omega0.  It is
trained on solutions the batched solver computes, and used through the batched
solver's warm start.  The KKT error decides: for each LP the prediction is used only
if its largest relative error (the three termination tests of Section 2, measured by
the solver at iteration 0) is below the cold start's; otherwise that LP starts cold.
KKT_omega (Section 2, restart criteria) is not the judge: its gap term is not
normalised, and the cold start of a transportation LP, (0, 0), has a zero dual
residual and a zero gap, so KKT_omega(cold) = omega ||b|| is below that of any
approximate prediction, whose gap |q'y - c'x| is on the scale of the objective.
evaluate reports how many predictions each judge would take.

Normalisation is per component: parameters and targets are standardised with the
training set's mean and standard deviation (floor 1e-6); omega is learned in log
space.
"""
from __future__ import annotations

import time

import numpy as np

from . import MLP, BatchSolver


def _init_params(n_in, hidden, n_out, seed):
    rng = np.random.default_rng(seed)
    out = []
    for fi, fo in ((n_in, hidden), (hidden, hidden), (hidden, n_out)):
        a = 1.0 / np.sqrt(fi)
        out.append(rng.uniform(-a, a, (fo, fi)).astype(np.float32))
        out.append(rng.uniform(-a, a, fo).astype(np.float32))
    return out


def solve_family(lps, tol, chunk=4096, **params):
    """Solves LPs of one family (all of the same sizes) with the batched solver, `chunk`
    per launch.  Returns x (N x n) and y (N x m) as float32 training targets, omega (N,),
    iterations (N,), status (N,) and the device seconds."""
    N = len(lps)
    X = np.empty((N, lps[0]["n"]), dtype=np.float32)
    Y = np.empty((N, lps[0]["m"]), dtype=np.float32)
    ws, its, sts, dev = [], [], [], 0.0
    for s in range(0, N, chunk):
        part = lps[s:s + chunk]
        with BatchSolver.from_lps(part, **params) as b:
            res = b.solve(tol=tol)
        dev += res[0]["device_ms"] * 1e-3
        for i, r in enumerate(res):
            X[s + i] = r["x"]
            Y[s + i] = r["y"]
            ws.append(r["omega"])
            its.append(r["iters"])
            sts.append(r["status"])
    return (X, Y, np.array(ws), np.array(its), np.array(sts), dev)


class WarmStart:
    def __init__(self, n_params, n, m, hidden=1024, max_batch=256, seed=0):
        self.n_params, self.n, self.m = n_params, n, m
        self.net = MLP(n_params, hidden, n + m + 1, max_batch)
        self.net.set_params(_init_params(n_params, hidden, n + m + 1, seed))
        self.max_batch = max_batch

    def _targets(self, X, Y, W, a, b):
        """Rows a..b of the targets (x, y, log omega) in float64."""
        return np.concatenate([np.asarray(X[a:b], np.float64), np.asarray(Y[a:b], np.float64),
                               np.log(np.maximum(W[a:b], 1e-300))[:, None]], axis=1)

    def fit(self, P, X, Y, W, epochs=30, batch=256, lr=1e-3, weight_decay=0.0, seed=0, block=2048):
        """Standardises parameters and targets with the training set's column means and
        standard deviations (two float64 passes over blocks of `block` rows, so that no
        float64 copy of the whole target matrix is made), then trains."""
        N = len(W)
        self.p_mu, self.p_sd = P.mean(0), np.maximum(P.std(0), 1e-6)
        cols = self.n + self.m + 1
        s1 = np.zeros(cols)
        for a in range(0, N, block):
            s1 += self._targets(X, Y, W, a, min(a + block, N)).sum(0)
        self.t_mu = s1 / N
        s2 = np.zeros(cols)
        for a in range(0, N, block):
            d = self._targets(X, Y, W, a, min(a + block, N)) - self.t_mu
            s2 += (d * d).sum(0)
        self.t_sd = np.maximum(np.sqrt(s2 / N), 1e-6)
        Tn = np.empty((N, cols), dtype=np.float32)
        for a in range(0, N, block):
            b = min(a + block, N)
            Tn[a:b] = (self._targets(X, Y, W, a, b) - self.t_mu) / self.t_sd
        self.net.load_data(((P - self.p_mu) / self.p_sd).astype(np.float32), Tn)
        del Tn
        t0 = time.perf_counter()
        losses, ms = self.net.train(epochs, min(batch, self.max_batch), lr, weight_decay, seed)
        return dict(losses=losses, train_device_s=ms * 1e-3, train_wall_s=time.perf_counter() - t0)

    def predict(self, P):
        self.net.load_data((np.asarray(P) - self.p_mu) / self.p_sd)
        Tn = self.net.forward(np.arange(len(P), dtype=np.int32))
        T = Tn.astype(np.float64) * self.t_sd + self.t_mu
        x0 = np.maximum(T[:, :self.n], 0.0)
        y0 = T[:, self.n:self.n + self.m]
        w0 = np.exp(T[:, -1])
        return x0, y0, w0

    def close(self):
        self.net.close()


def evaluate(model, lps, P, tols=(1e-4, 1e-8), budget=None, **params):
    """Cold start against the learned warm start (with the KKT fallback) on held-out LPs,
    one batched launch per solve.  Returns per tolerance the mean iterations and the
    times of both paths, and how many LPs used the prediction.

    The warm path's time counts everything it needs beyond the cold path: the MLP
    inference (host wall time of predict, transfers included), the two iteration-0
    launches of the KKT judge (device time), the warm-started solve (device time) and,
    with an iteration budget, the cold re-solve of every LP that did not converge within
    it (device time of one batched launch over those LPs).  The judge compares the
    largest relative error of the three tests for the prediction and the cold start; the
    count KKT_omega would accept is reported beside it.

    budget: iteration budget of a warm-started solve; an LP that has not converged
    within it falls back to a cold start, and its count is the budget plus the cold
    solve's iterations."""
    t0 = time.perf_counter()
    x0, y0, w0 = model.predict(P)
    predict_s = time.perf_counter() - t0
    out = {"predict_wall_s": predict_s}
    with BatchSolver.from_lps(lps, **params) as b:
        # an untimed cold run of 640 iterations (the autotuner's first slice and up to
        # eight timed ones) lets the batched solver choose its launch configuration, so
        # that both timed paths run with the same one
        b.solve(tol=0.0, max_iter=640, want_points=False)
        c0 = b.solve(tol=0.0, max_iter=0, want_points=False)
        p0 = b.solve(tol=0.0, max_iter=0, want_points=False, x0=list(x0), y0=list(y0), omega0=w0)
        judge_s = (c0[0]["device_ms"] + p0[0]["device_ms"]) * 1e-3
        k_cold = np.array([r["kkt_omega"] for r in c0])
        k_pred = np.array([r["kkt_omega"] for r in p0])
        e_cold = np.array([max(r["rel_primal"], r["rel_dual"], r["rel_gap"]) for r in c0])
        e_pred = np.array([max(r["rel_primal"], r["rel_dual"], r["rel_gap"]) for r in p0])
        use = e_pred < e_cold
        xs = [x0[i] if use[i] else np.zeros(lp["n"]) for i, lp in enumerate(lps)]
        ys = [y0[i] if use[i] else np.zeros(lp["m"]) for i, lp in enumerate(lps)]
        ws = np.where(use, w0, 0.0)
        for tol in tols:
            cold = b.solve(tol=tol, want_points=False)
            wkw = {} if budget is None else {"max_iter": int(budget)}
            warm = b.solve(tol=tol, want_points=False, x0=xs, y0=ys, omega0=ws, **wkw)
            ci = np.array([r["iters"] for r in cold])
            wi = np.array([r["iters"] for r in warm])
            warm_s = warm[0]["device_ms"] * 1e-3
            over = np.array([r["status"] != 0 for r in warm]) if budget is not None else np.zeros(len(lps), bool)
            fallback_s = 0.0
            if over.any():
                # the fallback's cold re-solves, timed as the warm path would run them
                with BatchSolver.from_lps([lp for lp, o in zip(lps, over) if o], **params) as bf:
                    rf = bf.solve(tol=tol, want_points=False)
                fallback_s = rf[0]["device_ms"] * 1e-3
                fi = iter(rf)
                warm = [next(fi) if o else w for w, o in zip(warm, over)]
                wi = np.where(over, wi + ci, wi)
            cold_s = cold[0]["device_ms"] * 1e-3
            warm_total = predict_s + judge_s + warm_s + fallback_s
            out[f"{tol:.0e}"] = dict(
                cold_iters_mean=float(ci.mean()), warm_iters_mean=float(wi.mean()),
                iters_ratio=float(ci.mean() / max(wi.mean(), 1e-9)),
                cold_device_s=cold_s, warm_device_s=warm_s, judge_device_s=judge_s,
                fallback_device_s=fallback_s, warm_total_s=warm_total,
                time_ratio=cold_s / max(warm_total, 1e-12),
                time_ratio_solve_only=cold_s / max(warm_s, 1e-12),
                cold_optimal=int(sum(r["status"] == 0 for r in cold)),
                warm_optimal=int(sum(r["status"] == 0 for r in warm)),
                warm_fewer_iters=int(np.sum(wi < ci)), warm_more_iters=int(np.sum(wi > ci)),
                fell_back_after_budget=int(over.sum()))
    out["used_prediction"] = int(use.sum())
    out["used_prediction_by_kkt_omega"] = int(np.sum(k_pred < k_cold))
    out["initial_kkt_omega_cold_median"] = float(np.median(k_cold))
    out["initial_kkt_omega_pred_median"] = float(np.median(k_pred))
    out["initial_err_cold_median"] = float(np.median(e_cold))
    out["initial_err_pred_median"] = float(np.median(e_pred))
    return out

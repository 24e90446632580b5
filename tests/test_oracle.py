"""Pins of the CPU oracle against facts fixed outside it (arXiv 2312.14832, Section 2).

Each test checks the oracle against something it does not compute itself: a library
routine (scipy.sparse products, numpy SVD, HiGHS), brute-force vertex enumeration,
closed forms (box-only LPs), planted optima built to satisfy complementarity,
or theorems about PDHG (fixed point, Fejer monotonicity in the M-norm,
Pock-Chambolle's norm bound, weak duality, Ruiz equilibration).
"""
import itertools
import json
import os

import numpy as np
import pytest
import scipy.sparse as sp

import lpgen
import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


def dense(lp):
    return sp.csr_matrix((lp["val"], lp["col_idx"], lp["row_ptr"]), shape=(lp["m"], lp["n"]))


# ---------------------------------------------------------------- products

@pytest.mark.parametrize("seed", [0, 1])
def test_spmv_matches_scipy(seed):
    lengths = [0, 1, 31, 32, 33, 0, 5, 200, 1, 64] * 3
    rp, ci, v = lpgen.random_csr(seed, len(lengths), 300, lengths, dist="wide")
    lp = dict(m=len(lengths), n=300, m1=0, row_ptr=rp, col_idx=ci, val=v)
    K = dense(lp)
    x = np.random.default_rng(seed).standard_normal(300)
    y = np.random.default_rng(seed + 7).standard_normal(len(lengths))
    np.testing.assert_allclose(oracle.spmv(lp, x), K @ x, rtol=1e-13, atol=1e-10)
    np.testing.assert_allclose(oracle.spmv_t(lp, y), K.T @ y, rtol=1e-13, atol=1e-10)


# ---------------------------------------------------------------- cone and projections

def test_proj_lambda_cases():
    inf = np.inf
    # both infinite -> {0}
    assert oracle.proj_lambda(3.0, -inf, inf) == 0.0
    assert oracle.proj_lambda(-3.0, -inf, inf) == 0.0
    # only u finite -> R^-
    assert oracle.proj_lambda(-2.0, -inf, 1.0) == -2.0
    assert oracle.proj_lambda(2.0, -inf, 1.0) == 0.0
    # only l finite -> R^+
    assert oracle.proj_lambda(2.0, 0.0, inf) == 2.0
    assert oracle.proj_lambda(-2.0, 0.0, inf) == 0.0
    # both finite -> R
    assert oracle.proj_lambda(-2.0, 0.0, 1.0) == -2.0
    assert oracle.proj_lambda(2.0, 0.0, 1.0) == 2.0


# ---------------------------------------------------------------- planted optima

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_planted_optimum_is_kkt_point(seed):
    lp = lpgen.planted_small(seed)
    p = oracle.kkt_parts(lp, lp["x_star"], lp["y_star"])
    scale = 1.0 + np.abs(lp["c"]).max() * 10.0 + np.abs(lp["q"]).max()
    assert np.sqrt(p["pres2"]) < 1e-11 * scale * np.sqrt(lp["m"])
    assert np.sqrt(p["dres2"]) < 1e-11 * scale * np.sqrt(lp["n"])
    assert abs(p["gap"]) < 1e-10 * (1 + abs(lp["obj_star"]))
    assert abs(p["pobj"] - lp["obj_star"]) < 1e-12 * (1 + abs(lp["obj_star"]))
    g = dense(lp).T @ lp["y_star"]
    lam = np.array([oracle.proj_lambda(d, a, b) for d, a, b in zip(lp["c"] - g, lp["l"], lp["u"])])
    np.testing.assert_allclose(lam, lp["lam_star"], atol=1e-12)


def test_planted_zipf_small_is_kkt_point():
    lp = lpgen.planted_zipf(seed=3, n=4000, m=2000, nnz=40000)
    p = oracle.kkt_parts(lp, lp["x_star"], lp["y_star"])
    assert np.sqrt(p["pres2"]) <= 1e-9 * (1 + np.linalg.norm(lp["q"]))
    assert np.sqrt(p["dres2"]) <= 1e-9 * (1 + np.linalg.norm(lp["c"]))
    assert abs(p["gap"]) <= 1e-9 * (1 + abs(p["pobj"]))


@pytest.mark.parametrize("seed", [0, 3])
def test_planted_optimum_is_pdhg_fixed_point(seed):
    lp = lpgen.planted_small(seed)
    for eta, omega in ((0.05, 1.0), (0.1, 0.3), (0.02, 4.0)):
        x, y = oracle.pdhg_step(lp, lp["x_star"], lp["y_star"], eta, omega)
        np.testing.assert_allclose(x, lp["x_star"], rtol=1e-12, atol=1e-11)
        np.testing.assert_allclose(y, lp["y_star"], rtol=1e-12, atol=1e-11)


def test_nonoptimal_point_moves():
    lp = lpgen.planted_small(0)
    x0 = lp["x_star"].copy()
    x0[lp["l"] > -np.inf] = lp["l"][lp["l"] > -np.inf]
    x, y = oracle.pdhg_step(lp, x0, lp["y_star"], 0.05, 1.0)
    assert np.linalg.norm(x - x0) > 1e-6


# ---------------------------------------------------------------- PDHG theory

def test_fejer_monotone_in_M_norm():
    """For PDHG on L(x,y) = c'x - y'Kx + q'y with tau = eta/omega, sigma = eta*omega and
    eta ||K|| < 1, ||z^t - z*||_M is nonincreasing with M = [[I/tau, K'], [K, I/sigma]]."""
    for seed in (1, 4):
        lp = lpgen.planted_small(seed)
        K = dense(lp)
        s = np.linalg.norm(K.toarray(), 2)
        for omega in (0.5, 2.0):
            eta = 0.95 / s
            tau, sig = eta / omega, eta * omega

            def mnorm(dx, dy):
                return dx @ dx / tau + dy @ dy / sig + 2.0 * (dy @ (K @ dx))

            rng = np.random.default_rng(seed)
            x = np.clip(rng.standard_normal(lp["n"]) * 5, lp["l"], lp["u"])
            y = rng.standard_normal(lp["m"])
            y[lp["m1"]:] = np.abs(y[lp["m1"]:])
            prev = mnorm(x - lp["x_star"], y - lp["y_star"])
            assert prev > 0
            for _ in range(200):
                x, y = oracle.pdhg_step(lp, x, y, eta, omega)
                cur = mnorm(x - lp["x_star"], y - lp["y_star"])
                assert cur <= prev * (1 + 1e-10) + 1e-10
                prev = cur


def test_weak_duality():
    """For x primal feasible and y in Y with c - K'y - lambda = 0: dual obj <= primal obj."""
    for seed in range(5):
        lp = lpgen.tiny_lp(seed, n=5, m1=1, m2=3)
        rng = np.random.default_rng(100 + seed)
        # a primal feasible x from a feasibility LP solved by HiGHS
        K = lp["K_dense"]
        from scipy.optimize import linprog
        res = linprog(np.zeros(lp["n"]), A_ub=-K[lp["m1"]:], b_ub=-lp["q"][lp["m1"]:],
                      A_eq=K[: lp["m1"]], b_eq=lp["q"][: lp["m1"]],
                      bounds=list(zip(lp["l"], lp["u"])), method="highs")
        assert res.status == 0
        x = res.x
        for _ in range(10):
            y = rng.standard_normal(lp["m"])
            y[lp["m1"]:] = np.abs(y[lp["m1"]:])
            p = oracle.kkt_parts(lp, x, y)
            assert p["dres2"] < 1e-20   # all bounds finite: Lambda = R, so lambda = c - K'y
            assert p["dobj"] <= p["pobj"] + 1e-9


# ---------------------------------------------------------------- restart rule

def test_restart_decision_conditions():
    d = oracle.restart_decision
    inf = float("inf")
    # condition 1: sufficient decay, <= is inclusive
    assert d(0.2, 1.0, inf, 10, 1000) == 1
    assert d(0.19, 1.0, 0.1, 10, 1000) == 1
    # condition 2: necessary decay and no local progress (strictly larger than previous)
    assert d(0.5, 1.0, 0.4, 10, 1000) == 2
    assert d(0.8, 1.0, 0.4, 10, 1000) == 2
    assert d(0.5, 1.0, 0.5, 10, 1000) == 0      # equal to previous: progress not lost
    assert d(0.5, 1.0, inf, 10, 1000) == 0      # first check of an inner loop
    assert d(0.81, 1.0, 0.4, 10, 1000) == 0     # not enough decay
    # condition 3: long inner loop t >= 0.36 k
    assert d(0.9, 1.0, 0.4, 36, 100) == 3
    assert d(0.9, 1.0, 0.4, 35, 100) == 0
    assert d(2.0, 1.0, inf, 64, 64) == 3        # first loop: t = k


def _lp2x2(l0):
    """K = [A; G] = [[1, 2], [3, -1]] (one equality row, one >= row), q = (4, 3), c = (1, 1),
    x_0 in [l0, inf), x_1 free."""
    return dict(m=2, n=2, m1=1, row_ptr=np.array([0, 2, 4]), col_idx=np.array([0, 1, 0, 1], dtype=np.int32),
                val=np.array([1.0, 2.0, 3.0, -1.0]), c=np.array([1.0, 1.0]), q=np.array([4.0, 3.0]),
                l=np.array([l0, -np.inf]), u=np.array([np.inf, np.inf]))


def test_kkt_omega_weights_by_hand():
    """KKT_omega (Section 2, restart criteria) at points worked out by hand: omega^2 weighs
    the primal residual, 1/omega^2 the dual residual, the gap enters unweighted.

    Point 1: x = (1, 1), y = (0.5, 2), x_0 in [0, inf).
      Kx = (3, 2): Ax - b = 3 - 4 = -1, [h - Gx]^+ = [3 - 2]^+ = 1          -> primal part 2
      K'y = (6.5, -1), c - K'y = (-5.5, 2); Lambda_0 = R^+ gives lambda_0 = 0,
      Lambda_1 = {0} gives lambda_1 = 0                                     -> dual part 34.25
      q'y = 8, l'lambda^+ = u'lambda^- = 0, c'x = 2                          -> gap 6
      KKT_2^2 = 4*2 + 34.25/4 + 36 = 52.5625 (KKT_2 = 7.25);  KKT_0.5^2 = 0.5 + 137 + 36 = 173.5
    Point 2: x = (1, 1), y = (0, 0.1), x_0 in [0.5, inf).
      primal part 2 as above; K'y = (0.3, -0.1), c - K'y = (0.7, 1.1), lambda = (0.7, 0)
      -> dual part 1.21; dual objective q'y + l_0 lambda_0 = 0.3 + 0.35 = 0.65, c'x = 2 -> gap -1.35
      KKT_2^2 = 8 + 0.3025 + 1.8225 = 10.125;  KKT_0.5^2 = 0.5 + 4.84 + 1.8225 = 7.1625
    A swapped weighting gives 173.5 at omega = 2 for point 1 (and 52.5625 at 0.5).
    """
    p = oracle.kkt_parts(_lp2x2(0.0), np.array([1.0, 1.0]), np.array([0.5, 2.0]))
    assert (p["pres2"], p["dres2"], p["pobj"], p["dobj"], p["gap"]) == (2.0, 34.25, 2.0, 8.0, 6.0)
    assert oracle.kkt_omega(p, 2.0) == pytest.approx(7.25, rel=1e-15)
    assert oracle.kkt_omega(p, 0.5) == pytest.approx(np.sqrt(173.5), rel=1e-15)
    p = oracle.kkt_parts(_lp2x2(0.5), np.array([1.0, 1.0]), np.array([0.0, 0.1]))
    assert p["pres2"] == 2.0 and p["pobj"] == 2.0
    assert p["dres2"] == pytest.approx(1.21, rel=1e-15)
    assert p["dobj"] == pytest.approx(0.65, rel=1e-15) and p["gap"] == pytest.approx(-1.35, rel=1e-15)
    assert oracle.kkt_omega(p, 2.0) == pytest.approx(np.sqrt(10.125), rel=1e-15)
    assert oracle.kkt_omega(p, 0.5) == pytest.approx(np.sqrt(7.1625), rel=1e-15)


def _lp1x1():
    """min x  s.t.  x = 3, x free: K = [1], m1 = 1, c = 1, q = 3."""
    return dict(m=1, n=1, m1=1, row_ptr=np.array([0, 1]), col_idx=np.array([0], dtype=np.int32),
                val=np.array([1.0]), c=np.array([1.0]), q=np.array([3.0]), l=np.array([-np.inf]),
                u=np.array([np.inf]))


def test_first_restart_and_primal_weight_by_hand():
    """Two PDHG steps with a check after each, worked out by hand (Section 2 updates,
    restart criteria; the primal-weight update is this build's reading S5).

    eta = 0.5, omega = 2, z^0 = (0, 0):
      x^1 = x^0 - (eta/omega)(c - K'y^0) = -0.25;  y^1 = y^0 + eta omega (q - K(2x^1 - x^0)) = 3.5
    First check (k = t = 1): the average of one iterate is that iterate, so the two KKT values
    tie and the candidate is the average (strict <).  KKT_2(z^0)^2 = 4*9 + 1/4 = 36.25;
    KKT_2(z^1)^2 = 4*3.25^2 + 2.5^2/4 + (10.5 + 0.25)^2 = 159.375 > 0.8^2 * 36.25, so neither
    decay condition holds and t >= 0.36 k (condition 3) restarts.  dx = 0.25, dy = 3.5:
      omega <- exp(theta log(dy/dx) + (1 - theta) log omega) = sqrt(14 * 2) = sqrt(28) (theta = 0.5),
      14 with theta = 1, 2 with theta = 0.
    The new anchor is KKT at z^1 with the new omega: 28*10.5625 + 6.25/28 + 115.5625.
    Relative tests at z^1: 3.25/(1+3), 2.5/(1+1), 10.75/(1 + 10.5 + 0.25).
    """
    lp = _lp1x1()
    kw = dict(tol=1e-12, max_iter=2, check_every=1, eta=0.5, omega0=2.0, scaling=0, log_cap=4)
    r = oracle.solve(lp, **kw)
    assert list(r["restart_iters"]) == [1] and r["checks"] == 2
    c0, c1 = r["log"]
    assert (c0["k"], c0["t"], c0["restart"], c0["candidate"]) == (1, 1, 3, 1)
    assert c0["omega"] == 2.0
    assert c0["kkt_cur"] == c0["kkt_avg"] == pytest.approx(np.sqrt(159.375), rel=1e-15)
    assert c0["kkt_anchor"] == pytest.approx(np.sqrt(36.25), rel=1e-15)
    assert (c0["rel_primal"], c0["rel_dual"]) == (0.8125, 1.25)
    assert c0["rel_gap"] == pytest.approx(10.75 / 11.75, rel=1e-15)
    assert (c1["k"], c1["t"]) == (2, 1)
    assert c1["omega"] == pytest.approx(np.sqrt(28.0), rel=1e-14)
    assert c1["kkt_anchor"] == pytest.approx(np.sqrt(28 * 10.5625 + 6.25 / 28 + 115.5625), rel=1e-14)
    assert r["omega"] == pytest.approx(np.sqrt(28.0), rel=1e-14)
    assert oracle.solve(lp, **dict(kw, omega_theta=1.0))["omega"] == pytest.approx(14.0, rel=1e-14)
    assert oracle.solve(lp, **dict(kw, omega_theta=0.0))["omega"] == pytest.approx(2.0, rel=1e-15)


def test_initial_primal_weight_by_hand():
    """Without a given omega0 the first primal weight is ||c|| / ||q|| = 1/3 (reading S4);
    eta = 0.5 then gives x^1 = -1.5, y^1 = 0.5/3 * (3 + 3) = 1, so the first check sees
    KKT_{1/3}(z^1)^2 = (1/9)(4.5)^2 + 9 * 0^2 + (3 + 1.5)^2 = 22.5 and KKT(z^0)^2 = 1 + 9 = 10."""
    r = oracle.solve(_lp1x1(), tol=1e-12, max_iter=1, check_every=1, eta=0.5, scaling=0, log_cap=2)
    c0 = r["log"][0]
    assert c0["omega"] == pytest.approx(1.0 / 3.0, rel=1e-15)
    assert c0["kkt_cur"] == pytest.approx(np.sqrt(22.5), rel=1e-15)
    assert c0["kkt_anchor"] == pytest.approx(np.sqrt(10.0), rel=1e-15)
    np.testing.assert_allclose(r["x_cur"], [-1.5], rtol=1e-15)
    np.testing.assert_allclose(r["y_cur"], [1.0], rtol=1e-15)


def test_restart_candidate_strict_rule():
    """Section 2: the candidate is the current iterate only when its KKT_omega is strictly
    smaller than the average's; a tie goes to the average (1)."""
    cand = oracle.restart_candidate
    assert cand(1.0, 1.0) == 1
    assert cand(0.5, 1.0) == 0
    assert cand(1.0, 0.5) == 1
    assert cand(np.nextafter(1.0, 0.0), 1.0) == 0
    assert cand(1.0, np.nextafter(1.0, 0.0)) == 1
    assert cand(0.0, 0.0) == 1
    assert cand(np.inf, np.inf) == 1
    assert cand(3.0, np.inf) == 0


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_threaded_step_is_the_serial_step(threads):
    """The CPU baseline's all-core PDHG step (K' built by a counting sort, columns and rows
    split over threads) performs orc_pdhg_step's operations in the same order: three
    steps from a random point give the same bits, with empty rows and columns present."""
    lengths = [0, 1, 31, 32, 33, 0, 5, 200, 1, 64] * 5
    rp, ci, v = lpgen.random_csr(21, len(lengths), 700, lengths, dist="wide")
    rng = np.random.default_rng(22)
    m, n = len(lengths), 700
    l = np.where(rng.random(n) < 0.5, -np.inf, -1.0)
    u = np.where(rng.random(n) < 0.5, np.inf, 2.0)
    lp = dict(m=m, n=n, m1=m // 3, row_ptr=rp, col_idx=ci, val=v, c=rng.standard_normal(n),
              q=rng.standard_normal(m), l=l, u=u)
    x = np.clip(rng.standard_normal(n), l, u)
    y = rng.standard_normal(m)
    y[m // 3:] = np.abs(y[m // 3:])
    T = oracle.ThreadedStep(lp, threads)
    xs, ys = x.copy(), y.copy()
    xp, yp = x.copy(), y.copy()
    for _ in range(3):
        xs, ys = oracle.pdhg_step(lp, xs, ys, 0.4, 1.3)
        T.step(xp, yp, 0.4, 1.3)
    np.testing.assert_array_equal(xp, xs)
    np.testing.assert_array_equal(yp, ys)


# ---------------------------------------------------------------- scaling

def test_ruiz_equilibrates():
    """Ruiz passes drive every row and column infinity norm to 1."""
    rp, ci, v = lpgen.random_csr(5, 60, 80, np.random.default_rng(5).integers(1, 20, 60), dist="wide")
    lp = dict(m=60, n=80, m1=0, row_ptr=rp, col_idx=ci, val=v)
    K = dense(lp).toarray()
    nz_cols = np.abs(K).max(axis=0) > 0
    vs, Dr, Dc = oracle.scale(lp, ruiz_iters=60, pock_chambolle=False)
    Ks = dense(dict(lp, val=vs)).toarray()
    np.testing.assert_allclose(np.abs(Ks).max(axis=1), 1.0, rtol=1e-9)
    np.testing.assert_allclose(np.abs(Ks).max(axis=0)[nz_cols], 1.0, rtol=1e-9)
    np.testing.assert_allclose(Ks, Dr[:, None] * K * Dc[None, :], rtol=1e-13, atol=0)


def test_pock_chambolle_norm_bound():
    """After the Pock-Chambolle pass (alpha = 1) the scaled matrix has ||K||_2 <= 1."""
    for seed in range(3):
        lp = lpgen.planted_small(seed)
        K = dense(lp).toarray()
        for ruiz in (0, 3, 10):
            vs, Dr, Dc = oracle.scale(lp, ruiz_iters=ruiz)
            Ks = dense(dict(lp, val=vs)).toarray()
            assert np.linalg.norm(Ks, 2) <= 1.0 + 1e-12
            np.testing.assert_allclose(Ks, Dr[:, None] * K * Dc[None, :], rtol=1e-13, atol=0)


def test_power_norm_matches_svd():
    lp = lpgen.planted_small(2)
    s = np.linalg.norm(dense(lp).toarray(), 2)
    est = oracle.power_norm(lp, iters=2000)
    assert est <= s * (1 + 1e-12)
    assert est >= s * (1 - 1e-6)
    est100 = oracle.power_norm(lp, iters=100)
    assert s * 0.9 < est100 <= s * (1 + 1e-12)


# ---------------------------------------------------------------- whole solves

def _vertex_enumeration(lp):
    K = lp["K_dense"]
    n, m1, m = lp["n"], lp["m1"], lp["m"]
    rows = [(K[i], lp["q"][i]) for i in range(m1, m)]
    rows += [(np.eye(n)[j], lp["l"][j]) for j in range(n)]
    rows += [(np.eye(n)[j], lp["u"][j]) for j in range(n)]
    best = np.inf
    for comb in itertools.combinations(range(len(rows)), n - m1):
        M = np.vstack([K[:m1]] + [rows[r][0] for r in comb])
        rhs = np.concatenate([lp["q"][:m1], [rows[r][1] for r in comb]])
        if abs(np.linalg.det(M)) < 1e-9:
            continue
        x = np.linalg.solve(M, rhs)
        if np.all(x >= lp["l"] - 1e-9) and np.all(x <= lp["u"] + 1e-9) and \
                np.all(K[m1:] @ x >= lp["q"][m1:] - 1e-9):
            best = min(best, float(lp["c"] @ x))
    return best


@pytest.mark.parametrize("seed", range(8))
def test_tiny_lp_matches_vertex_enumeration(seed):
    lp = lpgen.tiny_lp(seed, n=5, m1=1, m2=3)
    best = _vertex_enumeration(lp)
    assert np.isfinite(best)
    r = oracle.solve(lp, tol=1e-8, max_iter=2_000_000)
    assert r["status"] == oracle.STATUS_OPTIMAL
    assert abs(r["primal_obj"] - best) <= 1e-6 * (1 + abs(best))
    from scipy.optimize import linprog
    K = lp["K_dense"]
    ref = linprog(lp["c"], A_ub=-K[lp["m1"]:], b_ub=-lp["q"][lp["m1"]:], A_eq=K[: lp["m1"]],
                  b_eq=lp["q"][: lp["m1"]], bounds=list(zip(lp["l"], lp["u"])), method="highs")
    assert abs(ref.fun - best) <= 1e-7 * (1 + abs(best))


@pytest.mark.parametrize("seed,free_frac", [(0, 0.0), (1, 0.3)])
def test_box_only_closed_form(seed, free_frac):
    lp = lpgen.box_only(seed, n=50, free_frac=free_frac)
    r = oracle.solve(lp, tol=1e-10, max_iter=100000)
    assert r["status"] == oracle.STATUS_OPTIMAL
    c, l, u = lp["c"], lp["l"], lp["u"]
    fin = np.isfinite(l)
    want = np.where(c > 0, l, u)
    np.testing.assert_allclose(r["x"][fin & (c != 0)], want[fin & (c != 0)], rtol=0, atol=1e-9)
    obj = np.sum(np.minimum(c[fin] * l[fin], c[fin] * u[fin]))
    assert abs(r["primal_obj"] - obj) <= 1e-9 * (1 + abs(obj))
    assert r["eta"] == 1.0   # ||K|| = 0


@pytest.mark.parametrize("scaling", [0, 1])
def test_planted_small_converges_to_planted_objective(scaling):
    lp = lpgen.planted_small(0)
    K = dense(lp)
    for tol in (1e-4, 1e-8):
        r = oracle.solve(lp, tol=tol, scaling=scaling)
        assert r["status"] == oracle.STATUS_OPTIMAL
        # independent evaluation of the three tests of Section 2 with scipy
        x, y = r["x"], r["y"]
        # unscaling x = Dc * xt rounds, so bounds hold to a few ulps
        slack = 1e-15 * (1 + np.abs(x)) * 4
        assert np.all(x >= lp["l"] - slack) and np.all(x <= lp["u"] + slack)
        assert np.all(y[lp["m1"]:] >= 0)
        Kx = K @ x
        pr = np.concatenate([Kx[: lp["m1"]] - lp["q"][: lp["m1"]],
                             np.maximum(lp["q"][lp["m1"]:] - Kx[lp["m1"]:], 0)])
        d = lp["c"] - K.T @ y
        fl, fu = np.isfinite(lp["l"]), np.isfinite(lp["u"])
        lam = np.where(fl & fu, d, np.where(fl, np.maximum(d, 0), np.where(fu, np.minimum(d, 0), 0)))
        dobj = lp["q"] @ y + np.sum(np.where(lam > 0, np.where(fl, lp["l"], 0) * lam, 0)) \
            + np.sum(np.where(lam < 0, np.where(fu, lp["u"], 0) * lam, 0))
        pobj = lp["c"] @ x
        assert np.linalg.norm(pr) <= tol * (1 + np.linalg.norm(lp["q"])) * (1 + 1e-9)
        assert np.linalg.norm(d - lam) <= tol * (1 + np.linalg.norm(lp["c"])) * (1 + 1e-9)
        assert abs(dobj - pobj) <= tol * (1 + abs(dobj) + abs(pobj)) * (1 + 1e-9)
        if tol == 1e-8:
            assert abs(pobj - lp["obj_star"]) <= 1e-6 * abs(lp["obj_star"])


def test_restart_schedule_properties():
    lp = lpgen.planted_small(1)
    r = oracle.solve(lp, tol=1e-8, check_every=64)
    its = r["restart_iters"]
    assert len(its) == r["restarts"] > 0
    assert its[0] == 64            # first loop: t = k, so the first check restarts
    assert np.all(its % 64 == 0)
    assert np.all(np.diff(its) > 0)


def test_max_iter_zero_returns_initial_point():
    lp = lpgen.planted_small(0)
    r = oracle.solve(lp, tol=1e-8, max_iter=0)
    assert r["iters"] == 0 and r["status"] == oracle.STATUS_ITER_LIMIT
    np.testing.assert_array_equal(r["x"], np.clip(0.0, lp["l"], lp["u"]))
    np.testing.assert_array_equal(r["y"], 0.0)


def test_iteration_limit_not_multiple_of_check():
    lp = lpgen.planted_small(0)
    r = oracle.solve(lp, tol=0.0, max_iter=100)
    assert r["iters"] == 100 and r["status"] == oracle.STATUS_ITER_LIMIT


def test_golden_regression():
    """The oracle reproduces its committed record for the small planted LP (written by
    tests/golden/make_golden.py from the oracle alone)."""
    with open(os.path.join(HERE, "golden", "planted_small_seed0.json")) as f:
        g = json.load(f)
    lp = lpgen.planted_small(0)
    for rec in g["solves"]:
        r = oracle.solve(lp, tol=rec["tol"], scaling=rec["scaling"])
        assert r["iters"] == rec["iters"]
        assert list(map(int, r["restart_iters"])) == rec["restart_iters"]
        assert abs(r["primal_obj"] - rec["primal_obj"]) <= 1e-12 * abs(rec["primal_obj"])


# ---------------------------------------------------------------- warm-start network (oracle)

def test_mlp_oracle_gradients_match_finite_differences():
    """The plain (float64, no BF16) network's backward pass against central differences."""
    from oracle import mlp
    rng = np.random.default_rng(0)
    params = [p.astype(np.float64) for p in mlp.init_params(5, 7, 3, seed=1)]
    X = rng.standard_normal((4, 5))
    T = rng.standard_normal((4, 3))
    loss, grads = mlp.loss_and_grads(params, X, T, use_bf16=False)
    h = 1e-6
    for p, g in zip(params, grads):
        flat = p.reshape(-1)
        gf = g.reshape(-1)
        for i in range(0, flat.shape[0], max(1, flat.shape[0] // 9)):
            old = flat[i]
            flat[i] = old + h
            lp = mlp.loss_and_grads(params, X, T, use_bf16=False)[0]
            flat[i] = old - h
            lm = mlp.loss_and_grads(params, X, T, use_bf16=False)[0]
            flat[i] = old
            assert abs((lp - lm) / (2 * h) - gf[i]) <= 1e-6 * (1 + abs(gf[i]))


def test_bf16_rounding():
    from oracle import mlp
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 3.14159, -2.5e-3, 0.0], dtype=np.float32)
    r = mlp.bf16(vals)
    assert r[0] == 1.0 and r[1] == 1.0          # a tie rounds to even
    assert r[2] == 1.0 + 2 ** -7
    assert abs(r[3] - 3.140625) < 1e-12
    assert np.all(np.abs(r - vals) <= np.abs(vals) * 2 ** -8)


# ---------------------------------------------------------------- adaptive step rule
# (step_rule = 1: the rule of the cited PDLP paper, an option beside the constant eta)

def _norm_K(lp):
    K = dense(lp).toarray()
    return np.linalg.svd(K, compute_uv=False)[0] if K.size else 0.0


@pytest.mark.parametrize("seed", range(4))
def test_adaptive_step_below_one_over_norm_is_accepted(seed):
    """2|dy'K dx| <= 2||K|| ||dx|| ||dy|| <= ||K|| (omega ||dx||^2 + ||dy||^2/omega), so
    eta_max >= 1/||K||_2 for every attempt: a first step with eta < 1/||K||_2 is
    accepted from any point and any primal weight."""
    lp = lpgen.planted_small(seed)
    nk = _norm_K(lp)
    rng = np.random.default_rng(seed)
    for trial in range(3):
        x0 = rng.standard_normal(lp["n"]) * 3
        y0 = rng.standard_normal(lp["m"]) * 3
        w0 = float(np.exp(rng.uniform(-2, 2)))
        r = oracle.solve(lp, tol=0.0, max_iter=1, step_rule=1, eta=0.999 / nk, omega0=w0, x0=x0, y0=y0)
        assert r["iters"] == 1 and r["accepted"] == 1
        # the accepted step is the plain PDHG step of Section 2 with that eta
        xs, ys = oracle.pdhg_step(lp, np.clip(x0, lp["l"], lp["u"]),
                                  np.where(np.arange(lp["m"]) >= lp["m1"], np.maximum(y0, 0), y0),
                                  0.999 / nk, w0)
        np.testing.assert_allclose(r["x_cur"], xs, rtol=0, atol=1e-12 * (1 + np.abs(xs).max()))
        np.testing.assert_allclose(r["y_cur"], ys, rtol=0, atol=1e-12 * (1 + np.abs(ys).max()))


def test_adaptive_step_without_rows_grows_by_the_closed_form():
    """With no rows dy'K dx = 0, so every attempt is accepted and eta only grows:
    eta_s = eta_0 prod_{i=1..s} (1 + (i+1)^-0.6), eta_0 = 1 (K = 0).  The point still
    reaches the box optimum of the closed form."""
    lp = lpgen.box_only(3, n=40)
    r = oracle.solve(lp, tol=0.0, max_iter=10, step_rule=1)
    assert r["accepted"] == 10
    want = np.prod([1.0 + (i + 1.0) ** -0.6 for i in range(1, 11)])
    assert abs(r["eta"] - want) <= 1e-13 * want
    r = oracle.solve(lp, tol=1e-10, max_iter=100000, step_rule=1)
    assert r["status"] == oracle.STATUS_OPTIMAL
    c, l, u = lp["c"], lp["l"], lp["u"]
    np.testing.assert_allclose(r["x"], np.where(c > 0, l, u), rtol=0, atol=1e-9)


def test_adaptive_first_attempt_by_hand():
    """The adaptive rule's first attempt on min x s.t. x = 3 (x free), eta = 0.5,
    omega = 2, from z = 0, worked by hand (reading A1-A2): the attempt is the plain PDHG
    step, dx = -0.25, dy = 3.5, dy' K dx = -0.875; eta_max = (2 * 0.0625 + 12.25 / 2) /
    (2 * 0.875) = 25/7 >= 0.5, so the step is kept (s = 1, s + 1 = 2) and the next eta is
    min((1 - 2^-0.3) * 25/7, (1 + 2^-0.6) * 0.5) = (1 - 2^-0.3) * 25/7 = 0.6705..."""
    r = oracle.solve(_lp1x1(), tol=1e-12, max_iter=1, check_every=1, eta=0.5, omega0=2.0, scaling=0,
                     step_rule=1)
    assert r["accepted"] == 1
    np.testing.assert_allclose(r["x_cur"], [-0.25], rtol=1e-15)
    np.testing.assert_allclose(r["y_cur"], [3.5], rtol=1e-15)
    want = (1.0 - 2.0 ** -0.3) * 25.0 / 7.0
    assert want < (1.0 + 2.0 ** -0.6) * 0.5
    assert r["eta"] == pytest.approx(want, rel=1e-14)


def test_adaptive_rejection_and_cap_by_hand():
    """The rejection branch and the rejection cap on min x s.t. x = 3 (x free), worked by
    hand from the warm start x = 5, y = 0 with omega = 1 and eta = 3 (tau = sigma = 3):
    the attempt is x' = 5 - 3 * 1 = 2, y' = 3 * (3 - (2 * 2 - 5)) = 12, so dx = -3,
    dy = 12, dy' K dx = -36 and eta_max = (9 + 144) / 72 = 2.125 < 3.  With the default
    cap (64) the attempt is rejected: the point stays (5, 0), nothing is accepted, and the
    next eta is min((1 - 2^-0.3) * 2.125, (1 + 2^-0.6) * 3) = (1 - 2^-0.3) * 2.125 (s = 1,
    no step accepted yet).  With cap 0 the same attempt is kept: the point is (2, 12).
    This fails if a rejection moves the point, if the cap comparison is inverted or
    compares against the wrong count, or if the step size after a rejection is taken
    from the wrong branch."""
    kw = dict(tol=1e-12, max_iter=1, check_every=1, eta=3.0, omega0=1.0, scaling=0, step_rule=1)
    r = oracle.solve(_lp1x1(), x0=[5.0], y0=[0.0], **kw)
    assert r["accepted"] == 0
    np.testing.assert_array_equal(r["x_cur"], [5.0])
    np.testing.assert_array_equal(r["y_cur"], [0.0])
    want = (1.0 - 2.0 ** -0.3) * 2.125
    assert want < (1.0 + 2.0 ** -0.6) * 3.0
    assert r["eta"] == pytest.approx(want, rel=1e-14)
    r0 = oracle.solve(_lp1x1(), x0=[5.0], y0=[0.0], reject_cap=0, **kw)
    assert r0["accepted"] == 1
    np.testing.assert_allclose(r0["x_cur"], [2.0], rtol=1e-15)
    np.testing.assert_allclose(r0["y_cur"], [12.0], rtol=1e-15)
    assert r0["eta"] == pytest.approx(want, rel=1e-14)   # the next step size is the same either way


@pytest.mark.parametrize("seed", range(4))
def test_adaptive_tiny_lp_matches_vertex_enumeration(seed):
    lp = lpgen.tiny_lp(seed, n=5, m1=1, m2=3)
    best = _vertex_enumeration(lp)
    r = oracle.solve(lp, tol=1e-8, max_iter=2_000_000, step_rule=1)
    assert r["status"] == oracle.STATUS_OPTIMAL
    assert r["accepted"] <= r["iters"]
    assert abs(r["primal_obj"] - best) <= 1e-6 * (1 + abs(best))


@pytest.mark.parametrize("scaling", [0, 1])
def test_adaptive_planted_small_reaches_planted_objective(scaling):
    lp = lpgen.planted_small(0)
    r = oracle.solve(lp, tol=1e-8, scaling=scaling, step_rule=1)
    assert r["status"] == oracle.STATUS_OPTIMAL
    assert 0 < r["accepted"] <= r["iters"]
    assert abs(r["primal_obj"] - lp["obj_star"]) <= 1e-6 * abs(lp["obj_star"])
    x = r["x"]
    Kx = dense(lp) @ x
    pr = np.concatenate([Kx[: lp["m1"]] - lp["q"][: lp["m1"]], np.maximum(lp["q"][lp["m1"]:] - Kx[lp["m1"]:], 0)])
    assert np.linalg.norm(pr) <= 1e-8 * (1 + np.linalg.norm(lp["q"])) * (1 + 1e-9)


# ---------------------------------------------------------------- PageRank-shaped LP

def test_pagerank_lp_optimum_is_the_pagerank_vector():
    """The generator's x_star is the PageRank vector by its definition (the fixed point
    of x = damping S x + (1 - damping)/n with sum 1, reached here by plain power
    iteration on the link matrix), and the oracle's solution at 1e-8 is that vector."""
    lp = lpgen.pagerank(300, seed=1)
    n = lp["n"]
    # the link matrix from the LP's inequality rows: row i = e_i - damping S_i
    K = dense(lp).toarray()
    S = (np.eye(n) - K[1:n + 1]) / 0.85
    assert np.allclose(S.sum(axis=0), 1.0)            # column-stochastic
    x = np.full(n, 1.0 / n)
    for _ in range(500):
        x = 0.85 * S @ x + 0.15 / n
    assert abs(x.sum() - 1.0) < 1e-12
    np.testing.assert_allclose(lp["x_star"], x, rtol=1e-12, atol=0)
    for scaling in (0, 1):
        r = oracle.solve(lp, tol=1e-8, scaling=scaling)
        assert r["status"] == oracle.STATUS_OPTIMAL
        assert np.abs(r["x"] - x).max() <= 1e-5 * x.max()

"""Parity of the batched persistent solver (pdlp_batch_setup / pdlp_batch_solve) with
the CPU oracle, LP by LP.  Same tolerances as test_gpu_parity: relative 1e-10 on the
returned point after a fixed number of iterations (with the same restart count and
returned-point choice), relative 1e-6 on objectives at a tolerance (same iteration
count), 1e-13 * sum |K_ij x_j| on SpMV rows."""
import numpy as np
import pytest
import scipy.sparse as sp

import lpgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    from paper_2312_14832_b300 import build
    build.build()
    import paper_2312_14832_b300 as pk
    return pk


def mixed_batch():
    lps = lpgen.batch_planted(6, seed=100, n_lo=50, n_hi=1200)
    lps.append(lpgen.planted_small(3))
    lps.append(lpgen.box_only(4, n=70, free_frac=0.2))          # no rows at all
    lps.append(lpgen.planted_random(np.random.default_rng(9), 3, 4, 40, 60))   # tiny
    lps.append(lpgen.tiny_lp(2, n=5, m1=1, m2=3))
    return lps


def close_rel(a, b, rel):
    a, b = np.asarray(a), np.asarray(b)
    if b.size == 0:
        return
    scale = max(np.abs(b).max(), 1e-300)
    assert np.abs(a - b).max() <= rel * scale
    assert np.linalg.norm(a - b) <= rel * max(np.linalg.norm(b), 1e-300)


def decided_restarts(ref, restarts, floor=1e-9):
    """Restarts at checks whose decision rests on more than rounding noise: those before
    the first check at which the oracle's KKT_omega (current or average) has fallen below
    `floor` times its first anchor.  A tiny LP solved to machine precision has KKT values
    of ~1e-14 there, and which of two noise-level values is larger depends on summation
    order, so later decisions are not comparable.  Returns (the restarts before that check,
    True when the whole run stayed above the floor)."""
    log = ref["log"]
    scale = log[0]["kkt_anchor"] if log else 0.0
    cutoff = None
    for c in log:
        if min(c["kkt_cur"], c["kkt_avg"]) < floor * scale:
            cutoff = c["k"]
            break
    rs = np.asarray(restarts)
    return (rs if cutoff is None else rs[rs < cutoff]), cutoff is None


def fixed_iteration_batch():
    # the box-only LP is left out here: its residuals reach exactly zero, so a
    # tolerance of 0 is a tie that FP rounding may decide either way; it is covered
    # at nonzero tolerances below
    return [lp for lp in mixed_batch() if lp["m"] > 0]


@pytest.mark.parametrize("scaling", [0, 1])
def test_batch_iterates_after_1000(pk, scaling):
    lps = fixed_iteration_batch()
    with pk.BatchSolver.from_lps(lps, scaling=scaling) as b:
        res = b.solve(tol=0.0, max_iter=1000)
        restarts = [b.restarts(i) for i in range(len(lps))]
    for lp, r, rs in zip(lps, res, restarts):
        ref = oracle.solve(lp, tol=0.0, max_iter=1000, scaling=scaling, log_cap=4096)
        assert r["iters"] == ref["iters"] == 1000
        assert r["status"] == pk.ITER_LIMIT
        want, whole = decided_restarts(ref, ref["restart_iters"])
        got, _ = decided_restarts(ref, rs)
        np.testing.assert_array_equal(got, want)
        if whole:
            assert r["restarts"] == ref["restarts"]
            assert r["which"] == ref["which"]
        assert abs(r["eta"] - ref["eta"]) <= 1e-12 * ref["eta"]
        # omega is a function of ||x_c - x_anchor|| between nearly equal iterates: held to
        # 1e-9 while the run stays above the rounding floor, to 1e-6 for an LP whose later
        # restarts are decided on noise; the iterates themselves are held to 1e-10 below
        assert abs(r["omega"] - ref["omega"]) <= (1e-9 if whole else 1e-6) * ref["omega"]
        close_rel(r["x"], ref["x"], 1e-10)
        close_rel(r["y"], ref["y"], 1e-10)


@pytest.mark.parametrize("tol", [1e-4, 1e-8])
def test_batch_objectives_at_tolerance(pk, tol):
    lps = mixed_batch()
    with pk.BatchSolver.from_lps(lps) as b:
        res = b.solve(tol=tol, max_iter=500_000)
    for lp, r in zip(lps, res):
        ref = oracle.solve(lp, tol=tol, max_iter=500_000)
        assert r["status"] == ref["status"] == pk.OPTIMAL
        assert r["iters"] == ref["iters"]
        assert abs(r["primal_obj"] - ref["primal_obj"]) <= 1e-6 * (1 + abs(ref["primal_obj"]))
        assert max(r["rel_primal"], r["rel_dual"], r["rel_gap"]) <= tol


def test_batch_autotuner_keeps_the_result(pk):
    """The online autotuner (first solve of a handle) times its candidates on the solve's
    own iterations, resumed slice by slice, so the result is the untuned one up to
    summation order: same iteration counts, restart lists and returned-point choices,
    points within 1e-10.  The second solve keeps the choice without timing again."""
    lps = fixed_iteration_batch()
    with pk.BatchSolver.from_lps(lps) as b:
        tuned = b.solve(tol=0.0, max_iter=1000)
        info = b.info()
        tuned_rs = [b.restarts(i) for i in range(len(lps))]
        again = b.solve(tol=0.0, max_iter=1000)
        info2 = b.info()
    with pk.BatchSolver.from_lps(lps) as b:
        rule = b.solve(tol=0.0, max_iter=1000, batch_tune=1)
        rule_rs = [b.restarts(i) for i in range(len(lps))]
        assert b.info()["batch_tuned"] == 0
    assert info["batch_tuned"] >= 2, info
    assert info2["batch_tuned"] == 0
    k = info["batch_tuned"]
    assert all(g > 0 for g in info["tune_gbs"][:k])
    best = int(np.argmax(info["tune_gbs"][:k]))
    assert info2["batch_team"] == info["tune_team"][best]
    assert tuned[0]["launches"] == 2 + k and again[0]["launches"] == 1 and rule[0]["launches"] == 1
    for lp, a, b2, c, ra, rc in zip(lps, tuned, again, rule, tuned_rs, rule_rs):
        assert a["iters"] == b2["iters"] == c["iters"] == 1000
        ref = oracle.solve(lp, tol=0.0, max_iter=1000, log_cap=4096)
        want, whole = decided_restarts(ref, rc)
        np.testing.assert_array_equal(decided_restarts(ref, ra)[0], want)
        if whole:
            assert a["which"] == c["which"] and a["restarts"] == c["restarts"]
        close_rel(a["x"], c["x"], 1e-10)
        close_rel(a["y"], c["y"], 1e-10)
        close_rel(b2["x"], c["x"], 1e-10)


def test_batch_team_sizes_on_one_handle(pk):
    """Solves of one handle with different team sizes (each a CUDA graph of its own
    launch configuration) and back: every solve runs its iterations and gives the same
    point up to summation order."""
    lps = fixed_iteration_batch()[:6]
    with pk.BatchSolver.from_lps(lps) as b:
        runs = [b.solve(tol=0.0, max_iter=300, cluster_ctas=t) for t in (1, 2, 4, 2, 1)]
    for r in runs:
        assert all(x["iters"] == 300 for x in r)
        for a, c in zip(r, runs[0]):
            close_rel(a["x"], c["x"], 1e-10)
            close_rel(a["y"], c["y"], 1e-10)


def test_batch_ragged_iteration_limit_and_zero(pk):
    lps = fixed_iteration_batch()[:4]
    with pk.BatchSolver.from_lps(lps) as b:
        for iters in (0, 1, 100):
            res = b.solve(tol=0.0, max_iter=iters)
            for lp, r in zip(lps, res):
                ref = oracle.solve(lp, tol=0.0, max_iter=iters)
                assert r["iters"] == iters
                close_rel(r["x"], ref["x"], 1e-10)
                close_rel(r["y"], ref["y"], 1e-10)


def test_batch_block_diagonal_spmv(pk):
    lps = mixed_batch()
    x = [np.random.default_rng(i).standard_normal(lp["n"]) for i, lp in enumerate(lps)]
    with pk.BatchSolver.from_lps(lps) as b:
        got = b.spmv(np.concatenate(x))
    off = 0
    for lp, xi in zip(lps, x):
        K = sp.csr_matrix((lp["val"], lp["col_idx"], lp["row_ptr"]), shape=(lp["m"], lp["n"]))
        want = oracle.spmv(lp, xi)
        bound = 1e-13 * (abs(K) @ np.abs(xi)) + 1e-300
        assert np.all(np.abs(got[off:off + lp["m"]] - want) <= bound)
        off += lp["m"]


def test_batch_matches_single_solver(pk):
    lps = lpgen.batch_planted(3, seed=7, n_lo=200, n_hi=600)
    with pk.BatchSolver.from_lps(lps) as b:
        res = b.solve(tol=1e-6)
    for lp, r in zip(lps, res):
        with pk.Solver.from_lp(lp) as s:
            r1 = s.solve(tol=1e-6)
        assert r1["iters"] == r["iters"]
        close_rel(r["x"], r1["x"], 1e-10)


def test_batch_warm_start_matches_oracle(pk):
    lps = fixed_iteration_batch()[:5]
    rng = np.random.default_rng(3)
    x0 = [lp["x_star"] + 0.1 * rng.standard_normal(lp["n"]) if "x_star" in lp else rng.standard_normal(lp["n"])
          for lp in lps]
    y0 = [rng.standard_normal(lp["m"]) for lp in lps]
    w0 = np.array([0.5, 0.0, 2.0, 1.0, 0.0])
    with pk.BatchSolver.from_lps(lps) as b:
        res = b.solve(tol=0.0, max_iter=400, x0=x0, y0=y0, omega0=w0)
    for i, (lp, r) in enumerate(zip(lps, res)):
        ref = oracle.solve(lp, tol=0.0, max_iter=400, x0=x0[i], y0=y0[i], omega0=float(w0[i]))
        assert r["restarts"] == ref["restarts"]
        close_rel(r["x"], ref["x"], 1e-10)
        close_rel(r["y"], ref["y"], 1e-10)


@pytest.mark.parametrize("team,resident", [(2, 1), (2, 2), (8, 1), (8, 2), (16, 2), (1, 3), (4, 3)])
def test_cluster_team_iterates_after_1000(pk, team, resident):
    """Several CTAs (a thread-block cluster) share each LP, with the matrix streamed from
    global memory (resident=1), staged in shared memory (2), or the iterates themselves
    in global memory (3, one copy per LP): same iterates as the oracle."""
    lps = fixed_iteration_batch()
    with pk.BatchSolver.from_lps(lps, scaling=1) as b:
        res = b.solve(tol=0.0, max_iter=1000, cluster_ctas=team, resident=resident)
        info = b.info()
        assert info["batch_team"] == team
        if resident == 1:
            assert info["batch_resident"] == 0
        if team >= 8 and resident == 2:   # every slice fits once the LPs are cut 8 ways
            assert info["batch_resident"] == 1
        if resident == 3:
            assert info["batch_resident"] == 3
    for lp, r in zip(lps, res):
        ref = oracle.solve(lp, tol=0.0, max_iter=1000, scaling=1)
        assert r["iters"] == 1000 and r["status"] == pk.ITER_LIMIT
        assert r["restarts"] == ref["restarts"]
        assert r["which"] == ref["which"]
        assert abs(r["eta"] - ref["eta"]) <= 1e-12 * ref["eta"]
        assert abs(r["omega"] - ref["omega"]) <= 1e-6 * ref["omega"]
        close_rel(r["x"], ref["x"], 1e-10)
        close_rel(r["y"], ref["y"], 1e-10)


def test_resident_one_cta_per_lp(pk):
    """Small LPs whose whole matrix fits in one CTA's shared memory, one CTA each."""
    lps = [lp for lp in lpgen.batch_planted(8, seed=21, n_lo=40, n_hi=300) if lp["m"] > 0]
    lps.append(lpgen.tiny_lp(5, n=6, m1=2, m2=2))
    with pk.BatchSolver.from_lps(lps) as b:
        res = b.solve(tol=0.0, max_iter=700, cluster_ctas=1, resident=2)
        assert b.info()["batch_team"] == 1 and b.info()["batch_resident"] == 1
    for lp, r in zip(lps, res):
        ref = oracle.solve(lp, tol=0.0, max_iter=700)
        assert r["restarts"] == ref["restarts"]
        close_rel(r["x"], ref["x"], 1e-10)
        close_rel(r["y"], ref["y"], 1e-10)


@pytest.mark.parametrize("tol", [1e-4, 1e-8])
def test_cluster_single_small_lp_at_tolerance(pk, tol):
    """One LP, automatic team size (the whole cluster on one LP), against the oracle."""
    lp = lpgen.planted_small(0)
    ref = oracle.solve(lp, tol=tol)
    with pk.BatchSolver.from_lps([lp]) as b:
        for team, resident in ((0, 0), (4, 1), (1, 2)):
            r = b.solve(tol=tol, cluster_ctas=team, resident=resident)[0]
            assert r["status"] == ref["status"] == pk.OPTIMAL
            assert r["iters"] == ref["iters"]
            assert abs(r["primal_obj"] - ref["primal_obj"]) <= 1e-6 * abs(ref["primal_obj"])
            assert abs(r["primal_obj"] - lp["obj_star"]) <= 10 * tol * abs(lp["obj_star"])


def test_cluster_warm_start_and_rerun(pk):
    lps = fixed_iteration_batch()[:5]
    rng = np.random.default_rng(5)
    x0 = [rng.standard_normal(lp["n"]) for lp in lps]
    y0 = [rng.standard_normal(lp["m"]) for lp in lps]
    w0 = np.array([0.0, 1.5, 0.0, 0.7, 2.0])
    with pk.BatchSolver.from_lps(lps) as b:
        for _ in range(2):   # the queue counter resets itself between launches
            res = b.solve(tol=0.0, max_iter=300, x0=x0, y0=y0, omega0=w0, cluster_ctas=4, resident=2)
            for i, (lp, r) in enumerate(zip(lps, res)):
                ref = oracle.solve(lp, tol=0.0, max_iter=300, x0=x0[i], y0=y0[i], omega0=float(w0[i]))
                close_rel(r["x"], ref["x"], 1e-10)
                close_rel(r["y"], ref["y"], 1e-10)


@pytest.mark.parametrize("scaling,resident", [(0, 1), (1, 0), (1, 3)])
def test_two_stage_tail_matches_oracle(pk, scaling, resident):
    """batch_tail_iters: every LP stops at the first check after 192 iterations and the
    unfinished ones continue in a second launch on teams; the point after 1000
    iterations is the oracle's (the continuation changes only summation order)."""
    lps = fixed_iteration_batch()
    with pk.BatchSolver.from_lps(lps, scaling=scaling) as b:
        res = b.solve(tol=0.0, max_iter=1000, batch_tail_iters=192, resident=resident)
        info = b.info()
    assert info["batch_resumed"] == len(lps)
    for lp, r in zip(lps, res):
        ref = oracle.solve(lp, tol=0.0, max_iter=1000, scaling=scaling)
        assert r["iters"] == 1000 and r["status"] == pk.ITER_LIMIT
        assert r["restarts"] == ref["restarts"] and r["which"] == ref["which"]
        assert abs(r["omega"] - ref["omega"]) <= 1e-6 * ref["omega"]
        close_rel(r["x"], ref["x"], 1e-10)
        close_rel(r["y"], ref["y"], 1e-10)


def test_two_stage_tail_at_tolerance(pk):
    lps = mixed_batch()
    with pk.BatchSolver.from_lps(lps) as b:
        res = b.solve(tol=1e-8, max_iter=500_000, batch_tail_iters=256)
        resumed = b.info()["batch_resumed"]
    assert resumed > 0
    for lp, r in zip(lps, res):
        ref = oracle.solve(lp, tol=1e-8, max_iter=500_000)
        assert r["status"] == ref["status"] == pk.OPTIMAL
        assert r["iters"] == ref["iters"]
        assert abs(r["primal_obj"] - ref["primal_obj"]) <= 1e-6 * (1 + abs(ref["primal_obj"]))


def _check_point(lp, x, y, tol):
    rp, rd, rg = oracle.relative_errors(lp, x, y)
    assert max(rp, rd, rg) <= tol * (1 + 1e-6), (rp, rd, rg)


@pytest.mark.parametrize("team,resident", [(1, 0), (4, 0), (1, 3), (4, 3)])
def test_batch_mixed_precision_at_1e4(pk, team, resident):
    """FP32 iterations with FP64 checks (precision = MIXED): every returned point passes
    the tests of Section 2 (re-evaluated by the oracle's KKT routine) and its objective
    agrees with the FP64 oracle within the requested accuracy (1e-3 relative at 1e-4,
    as for the single-LP mixed precision)."""
    lps = mixed_batch()
    with pk.BatchSolver.from_lps(lps, precision=pk.MIXED) as b:
        res = b.solve(tol=1e-4, max_iter=500_000, cluster_ctas=team, resident=resident)
    assert sum(r["fp32_iters"] for r in res) > 0
    for lp, r in zip(lps, res):
        ref = oracle.solve(lp, tol=1e-4, max_iter=500_000)
        assert r["status"] == pk.OPTIMAL
        assert r["fp32_iters"] <= r["iters"]
        _check_point(lp, r["x"], r["y"], 1e-4)
        assert abs(r["primal_obj"] - ref["primal_obj"]) <= 1e-3 * (1 + abs(ref["primal_obj"]))


def test_batch_mixed_precision_refines_to_1e8(pk):
    lps = mixed_batch()
    with pk.BatchSolver.from_lps(lps, precision=pk.MIXED) as b:
        res = b.solve(tol=1e-8, max_iter=500_000)
        resumed = b.info()["batch_resumed"]
    assert resumed > 0                                   # FP64 refinement ran
    assert any(0 < r["fp32_iters"] < r["iters"] for r in res)
    for lp, r in zip(lps, res):
        ref = oracle.solve(lp, tol=1e-8, max_iter=500_000)
        assert r["status"] == pk.OPTIMAL
        _check_point(lp, r["x"], r["y"], 1e-8)
        assert abs(r["primal_obj"] - ref["primal_obj"]) <= 1e-6 * (1 + abs(ref["primal_obj"]))


def test_batch_mixed_precision_iteration_limit(pk):
    lps = fixed_iteration_batch()[:4]
    with pk.BatchSolver.from_lps(lps, precision=pk.MIXED) as b:
        res = b.solve(tol=0.0, max_iter=300, mixed_switch_tol=1e-30)
    for r in res:
        assert r["iters"] == 300 and r["status"] == pk.ITER_LIMIT and r["fp32_iters"] == 300
        assert np.all(np.isfinite(r["x"])) and np.all(np.isfinite(r["y"]))


def test_global_iterates_for_an_lp_too_large_for_shared_memory(pk):
    """x and y of this LP (n + m > 30000) do not fit in one CTA's shared memory: the
    batch keeps them in global memory (automatic) and still matches the oracle."""
    lps = [lpgen.planted_random(np.random.default_rng(31), 6000, 9000, 24000, 60000)]
    lps.append(lpgen.planted_small(5))
    with pk.BatchSolver.from_lps(lps, scaling=1) as b:
        res = b.solve(tol=0.0, max_iter=400)
        assert b.info()["batch_resident"] == 3
        res_t = b.solve(tol=1e-6, max_iter=200_000, cluster_ctas=8)
    for lp, r, rt in zip(lps, res, res_t):
        ref = oracle.solve(lp, tol=0.0, max_iter=400, scaling=1)
        assert r["restarts"] == ref["restarts"]
        close_rel(r["x"], ref["x"], 1e-10)
        close_rel(r["y"], ref["y"], 1e-10)
        reft = oracle.solve(lp, tol=1e-6, max_iter=200_000, scaling=1)
        assert rt["status"] == reft["status"] == pk.OPTIMAL and rt["iters"] == reft["iters"]

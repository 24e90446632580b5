"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Tolerances (derived from FP64 rounding of the sums and of the iteration):
  * SpMV: |gpu - oracle| <= 1e-13 * sum_j |K_ij x_j| per row (different summation
    order only; FP64 rounding is ~1e-16 per term).
  * iterates after a fixed number of PDHG iterations: relative 1e-10 in the 2-norm
    and elementwise against 1e-10 * max |reference|.
  * objectives at a tolerance: relative 1e-6.
"""
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


def dense(lp):
    return sp.csr_matrix((lp["val"], lp["col_idx"], lp["row_ptr"]), shape=(lp["m"], lp["n"]))


def close_rel(a, b, rel):
    a = np.asarray(a)
    b = np.asarray(b)
    if b.size == 0:
        return
    scale = max(np.abs(b).max(), 1e-300)
    err = np.abs(a - b).max()
    assert err <= rel * scale, f"max abs err {err:.3e} > {rel:.1e} * {scale:.3e}"
    assert np.linalg.norm(a - b) <= rel * max(np.linalg.norm(b), 1e-300)


# ---------------------------------------------------------------- SpMV

LENGTH_REGIMES = {
    "mixed": [0, 1, 31, 32, 33, 0, 5, 200, 1, 64] * 7 + [3],
    "long": [10000, 1, 2, 4500, 0, 33, 700, 65, 64, 63] * 4,
    "uniform": [7] * 1000 + [0] * 17,
    "empty_rows": [0] * 50,
}


@pytest.mark.parametrize("regime", list(LENGTH_REGIMES))
@pytest.mark.parametrize("tile", [0, 8, 64])
def test_spmv_matches_oracle(pk, regime, tile):
    lengths = LENGTH_REGIMES[regime]
    n = 12000
    rp, ci, v = lpgen.random_csr(11, len(lengths), n, lengths, dist="wide")
    m = len(lengths)
    lp = dict(m=m, n=n, m1=m // 3, row_ptr=rp, col_idx=ci, val=v, c=np.zeros(n), q=np.zeros(m),
              l=np.full(n, -np.inf), u=np.full(n, np.inf))
    rng = np.random.default_rng(3)
    x = rng.standard_normal(n)
    y = rng.standard_normal(m)
    K = dense(lp)
    with pk.Solver.from_lp(lp, tile_slots=tile) as s:
        for _ in range(2):   # twice: split-chunk counters must be back at zero
            gx = s.spmv(x)
            gy = s.spmv(y, transpose=True)
            ref_x = oracle.spmv(lp, x)
            ref_y = oracle.spmv_t(lp, y)
            bx = abs(K) @ np.abs(x)
            by = abs(K).T @ np.abs(y)
            assert np.all(np.abs(gx - ref_x) <= 1e-13 * bx + 1e-300)
            assert np.all(np.abs(gy - ref_y) <= 1e-13 * by + 1e-300)


@pytest.mark.parametrize("regime", list(LENGTH_REGIMES))
@pytest.mark.parametrize("tile", [8, 64])
def test_staged_stream_spmv_bit_identical(pk, regime, tile):
    """The value/index stream staged in shared memory by bulk copies (spmv_stage 2: two
    8-slot buffers per warp, 3: three) gives the same bits as the coalesced global loads
    (spmv_stage 1) for the same task plan, and matches the oracle; ragged tasks (slot
    counts not multiples of 8), split chunks and empty rows included."""
    lengths = LENGTH_REGIMES[regime]
    n = 12000
    rp, ci, v = lpgen.random_csr(13, len(lengths), n, lengths, dist="wide")
    m = len(lengths)
    lp = dict(m=m, n=n, m1=m // 3, row_ptr=rp, col_idx=ci, val=v, c=np.zeros(n), q=np.zeros(m),
              l=np.full(n, -np.inf), u=np.full(n, np.inf))
    rng = np.random.default_rng(4)
    x = rng.standard_normal(n)
    y = rng.standard_normal(m)
    K = dense(lp)
    outs = {}
    for stage in (1, 2, 3):
        for batch in (4, 8):
            with pk.Solver.from_lp(lp, tile_slots=tile, spmv_batch=batch, spmv_stage=stage) as s:
                for _ in range(2):
                    gx = s.spmv(x)
                    gy = s.spmv(y, transpose=True)
                outs[(stage, batch)] = (gx, gy)
    for (stage, batch), (gx, gy) in outs.items():
        np.testing.assert_array_equal(gx, outs[(1, batch)][0])
        np.testing.assert_array_equal(gy, outs[(1, batch)][1])
        assert np.all(np.abs(gx - oracle.spmv(lp, x)) <= 1e-13 * (abs(K) @ np.abs(x)) + 1e-300)
        assert np.all(np.abs(gy - oracle.spmv_t(lp, y)) <= 1e-13 * (abs(K).T @ np.abs(y)) + 1e-300)


def test_spmv_scaled_roundtrip(pk):
    lp = lpgen.planted_zipf(seed=5, n=6000, m=3000, nnz=60000)
    x = np.random.default_rng(1).standard_normal(lp["n"])
    K = dense(lp)
    with pk.Solver.from_lp(lp, scaling=1) as s:
        gx = s.spmv(x)
    bx = abs(K) @ np.abs(x)
    assert np.all(np.abs(gx - K @ x) <= 1e-12 * bx + 1e-300)


# ---------------------------------------------------------------- iterates

def compare_logs(got, ref, rel=1e-8):
    """Per-check records: iteration counts, restart conditions and candidate choices
    identical; omega within rel.  The KKT_omega values and the relative tests are norms of
    residuals: the points agree to ~1e-15 of their magnitude, so a residual carries an
    absolute error of ~1e-15 of the problem's scale however small it gets (the gap is a
    difference of two objectives).  They are compared within rel plus 1e-12 of that
    scale: the largest KKT_omega of the log for the KKT values, and 1 for the relative
    tests, which are already divided by 1 + the norms of the data."""
    assert len(got) == len(ref)
    kscale = max(max(o["kkt_anchor"], o["kkt_cur"], o["kkt_avg"]) for o in ref) if ref else 0.0
    for g, o in zip(got, ref):
        assert (g["k"], g["t"], g["restart"], g["candidate"]) == (o["k"], o["t"], o["restart"], o["candidate"])
        assert abs(g["omega"] - o["omega"]) <= rel * o["omega"], (g, o)
        for f in ("kkt_cur", "kkt_avg", "kkt_anchor"):
            assert abs(g[f] - o[f]) <= rel * abs(o[f]) + 1e-12 * kscale, (f, g, o)
        for f in ("rel_primal", "rel_dual", "rel_gap"):
            assert abs(g[f] - o[f]) <= rel * abs(o[f]) + 1e-12, (f, g, o)


def _compare_iterates(pk, lp, iters, engine=0, **params):
    """engine 1: kernels launched per iteration (CUDA graphs); 2: the persistent engine
    (one launch of the batched kernel on a thread-block cluster)."""
    ref = oracle.solve(lp, tol=0.0, max_iter=iters, log_cap=4096, **params)
    with pk.Solver.from_lp(lp, scaling=params.get("scaling", 0), engine=engine) as s:
        r = s.solve(tol=0.0, max_iter=iters)
        compare_logs(s.log(), ref["log"])
        if engine == 2:
            assert r["launches"] == 1
        assert r["iters"] == ref["iters"] == iters
        assert r["status"] == pk.ITER_LIMIT
        np.testing.assert_array_equal(s.restarts(), ref["restart_iters"])
        xc, yc = s.iterate(0)
        xa, ya = s.iterate(1)
        close_rel(xc, ref["x_cur"], 1e-10)
        close_rel(yc, ref["y_cur"], 1e-10)
        close_rel(xa, ref["x_avg"], 1e-10)
        close_rel(ya, ref["y_avg"], 1e-10)
        assert abs(r["omega"] - ref["omega"]) <= 1e-10 * ref["omega"]
        assert abs(r["eta"] - ref["eta"]) <= 1e-12 * ref["eta"]
        assert r["which"] == ref["which"]
        close_rel(r["x"], ref["x"], 1e-10)
    return r, ref


ENGINES = [1, 2]


@pytest.mark.parametrize("engine", ENGINES)
def test_first_restart_and_primal_weight_by_hand(pk, engine):
    """min x s.t. x = 3 (x free), eta = 0.5, omega0 = 2, a check after every step.  By hand:
    z^1 = (-0.25, 3.5); at the first check the current iterate and the average coincide,
    so the candidate is the average (a tie, strict rule of Section 2); condition 3
    restarts; omega becomes sqrt(2 * 3.5 / 0.25) = sqrt(28); KKT_2(z^1)^2 = 159.375 and
    KKT_2(z^0)^2 = 36.25.  The oracle's test of the same case derives every number."""
    lp = dict(m=1, n=1, m1=1, row_ptr=np.array([0, 1]), col_idx=np.array([0], dtype=np.int32),
              val=np.array([1.0]), c=np.array([1.0]), q=np.array([3.0]), l=np.array([-np.inf]),
              u=np.array([np.inf]))
    with pk.Solver.from_lp(lp, engine=engine, check_every=1, eta=0.5) as s:
        r = s.solve(tol=1e-12, max_iter=2, omega0=2.0)
        log = s.log()
        assert list(s.restarts()) == [1]
    assert r["iters"] == 2 and len(log) == 2
    assert (log[0]["k"], log[0]["t"], log[0]["restart"], log[0]["candidate"]) == (1, 1, 3, 1)
    assert log[0]["kkt_cur"] == log[0]["kkt_avg"]
    assert log[0]["kkt_cur"] == pytest.approx(np.sqrt(159.375), rel=1e-14)
    assert log[0]["kkt_anchor"] == pytest.approx(np.sqrt(36.25), rel=1e-14)
    assert r["omega"] == pytest.approx(np.sqrt(28.0), rel=1e-14)
    assert log[1]["omega"] == pytest.approx(np.sqrt(28.0), rel=1e-14)
    ref = oracle.solve(lp, tol=1e-12, max_iter=2, check_every=1, eta=0.5, omega0=2.0, log_cap=4)
    compare_logs(log, ref["log"], rel=1e-14)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("scaling", [0, 1])
def test_iterates_after_1000_small_planted(pk, seed, scaling, engine):
    _compare_iterates(pk, lpgen.planted_small(seed), 1000, engine=engine, scaling=scaling)


@pytest.mark.parametrize("stage", [2, 3])
@pytest.mark.parametrize("seed", [0, 1])
def test_iterates_after_1000_staged_stream(pk, seed, stage):
    """The kernels launched per iteration with the staged value/index stream."""
    lp = lpgen.planted_small(seed)
    ref = oracle.solve(lp, tol=0.0, max_iter=1000, scaling=1, log_cap=4096)
    with pk.Solver.from_lp(lp, scaling=1, engine=1, spmv_stage=stage, tile_slots=8) as s:
        r = s.solve(tol=0.0, max_iter=1000)
        compare_logs(s.log(), ref["log"])
        np.testing.assert_array_equal(s.restarts(), ref["restart_iters"])
        xc, yc = s.iterate(0)
    close_rel(xc, ref["x_cur"], 1e-10)
    close_rel(yc, ref["y_cur"], 1e-10)
    close_rel(r["x"], ref["x"], 1e-10)


def test_iterates_after_1000_zipf(pk):
    lp = lpgen.planted_zipf(seed=2, n=20000, m=10000, nnz=200000)
    _compare_iterates(pk, lp, 1000, scaling=1)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("iters", [0, 1, 63, 64, 100])
def test_iteration_counts_and_ragged_intervals(pk, iters, engine):
    _compare_iterates(pk, lpgen.planted_small(4), iters, engine=engine)


@pytest.mark.parametrize("engine", ENGINES)
def test_box_only_lp(pk, engine):
    lp = lpgen.box_only(3, n=100, free_frac=0.2)
    ref = oracle.solve(lp, tol=1e-10, max_iter=100000)
    with pk.Solver.from_lp(lp, engine=engine) as s:
        r = s.solve(tol=1e-10, max_iter=100000)
    assert r["status"] == pk.OPTIMAL and r["iters"] == ref["iters"]
    close_rel(r["x"], ref["x"], 1e-12)
    assert r["eta"] == 1.0


@pytest.mark.parametrize("engine", ENGINES)
def test_warm_start_matches_oracle(pk, engine):
    lp = lpgen.planted_small(6)
    rng = np.random.default_rng(0)
    x0 = lp["x_star"] + 0.1 * rng.standard_normal(lp["n"])
    y0 = lp["y_star"] + 0.1 * rng.standard_normal(lp["m"])
    ref = oracle.solve(lp, tol=0.0, max_iter=500, x0=x0, y0=y0)
    with pk.Solver.from_lp(lp, engine=engine) as s:
        r = s.solve(x0=x0, y0=y0, tol=0.0, max_iter=500)
        xc, yc = s.iterate(0)
    close_rel(xc, ref["x_cur"], 1e-10)
    close_rel(yc, ref["y_cur"], 1e-10)


# ---------------------------------------------------------------- solves to tolerance

@pytest.mark.parametrize("tol", [1e-4, 1e-8])
@pytest.mark.parametrize("scaling", [0, 1])
@pytest.mark.parametrize("engine", ENGINES)
def test_objective_at_tolerance(pk, tol, scaling, engine):
    lp = lpgen.planted_small(0)
    ref = oracle.solve(lp, tol=tol, scaling=scaling)
    with pk.Solver.from_lp(lp, scaling=scaling, engine=engine) as s:
        r = s.solve(tol=tol)
    assert r["status"] == pk.OPTIMAL
    assert r["iters"] == ref["iters"]
    assert abs(r["primal_obj"] - ref["primal_obj"]) <= 1e-6 * abs(ref["primal_obj"])
    assert abs(r["dual_obj"] - ref["dual_obj"]) <= 1e-6 * abs(ref["dual_obj"])
    assert max(r["rel_primal"], r["rel_dual"], r["rel_gap"]) <= tol
    if tol == 1e-8:
        assert abs(r["primal_obj"] - lp["obj_star"]) <= 1e-6 * abs(lp["obj_star"])


@pytest.mark.parametrize("seed", range(4))
def test_tiny_lp_objective(pk, seed):
    lp = lpgen.tiny_lp(seed, n=5, m1=1, m2=3)
    ref = oracle.solve(lp, tol=1e-8, max_iter=2_000_000)
    with pk.Solver.from_lp(lp) as s:
        r = s.solve(tol=1e-8, max_iter=2_000_000)
    assert r["status"] == pk.OPTIMAL
    assert abs(r["primal_obj"] - ref["primal_obj"]) <= 1e-6 * (1 + abs(ref["primal_obj"]))


@pytest.mark.parametrize("engine", ENGINES)
def test_solves_are_deterministic(pk, engine):
    lp = lpgen.planted_zipf(seed=7, n=8000, m=4000, nnz=80000)
    with pk.Solver.from_lp(lp, scaling=1, engine=engine) as s:
        a = s.solve(tol=0.0, max_iter=700)
        b = s.solve(tol=0.0, max_iter=700)
        np.testing.assert_array_equal(a["x"], b["x"])
        np.testing.assert_array_equal(a["y"], b["y"])


def test_invalid_inputs_are_rejected(pk):
    lp = lpgen.planted_small(0)
    bad = dict(lp, col_idx=lp["col_idx"].copy())
    bad["col_idx"][3] = lp["n"]
    with pytest.raises(pk.SolverError):
        pk.Solver.from_lp(bad)
    bad = dict(lp, l=lp["l"].copy())
    bad["l"][0] = 20.0   # l > u
    with pytest.raises(pk.SolverError):
        pk.Solver.from_lp(bad)
    bad = dict(lp, val=lp["val"].copy())
    bad["val"][0] = np.nan
    with pytest.raises(pk.SolverError):
        pk.Solver.from_lp(bad)


@pytest.mark.parametrize("scaling", [0, 1])
def test_bound_duals(pk, scaling):
    """pdlp_bound_duals: lambda = proj_Lambda(c - K'y) on the original problem, for any y
    (the oracle's projection applied to a scipy product), and at the solution the
    reduced costs that the dual residual test of Section 2 measures."""
    import scipy.sparse as sp
    lp = lpgen.planted_small(4)
    K = sp.csr_matrix((lp["val"], lp["col_idx"], lp["row_ptr"]), shape=(lp["m"], lp["n"]))
    rng = np.random.default_rng(2)
    y = rng.standard_normal(lp["m"])
    with pk.Solver.from_lp(lp, scaling=scaling) as s:
        lam = s.bound_duals(y)
        r = s.solve(tol=1e-8)
        lam_sol = s.bound_duals(r["y"])
    d = lp["c"] - K.T @ y
    want = np.array([oracle.proj_lambda(dj, lj, uj) for dj, lj, uj in zip(d, lp["l"], lp["u"])])
    bound = 1e-13 * (np.abs(lp["c"]) + abs(K).T @ np.abs(y)) + 1e-300
    near = np.abs(d) <= bound          # sign decided by rounding: either side is right
    assert np.all((np.abs(lam - want) <= bound) | near)
    rd = np.linalg.norm(lp["c"] - K.T @ r["y"] - lam_sol) / (1 + np.linalg.norm(lp["c"]))
    assert rd <= 1e-8 * (1 + 1e-6)


def test_engine_selection(pk):
    """The persistent engine is chosen automatically for a small FP64 LP, not with the
    adaptive rule, a time limit or mixed precision, and engine 2 is refused where it
    cannot run."""
    lp = lpgen.planted_small(1)
    with pk.Solver.from_lp(lp) as s:
        assert s.solve(tol=1e-4)["launches"] == 1
        assert s.solve(tol=1e-4, engine=1)["launches"] > 1
        assert s.solve(tol=1e-4, time_limit_s=100.0)["launches"] > 1
        assert s.solve(tol=1e-4, step_rule=1)["launches"] > 1
        with pytest.raises(pk.SolverError):
            s.solve(tol=1e-4, engine=2, step_rule=1)
    with pk.Solver.from_lp(lp, precision=pk.MIXED) as s:
        assert s.solve(tol=1e-4)["launches"] > 1
    big = lpgen.planted_zipf(seed=1, n=200000, m=100000, nnz=2000000)
    with pytest.raises(pk.SolverError):
        pk.Solver.from_lp(big, engine=2)

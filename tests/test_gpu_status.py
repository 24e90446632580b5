"""Solve outcomes other than OPTIMAL and ITER_LIMIT, through the C ABI.

The failures are made on the host, as parameters: a time limit shorter than one check
interval, and a step size so large that the iterates overflow.  Neither faults the GPU:
the time limit is read by the host between check intervals, and an overflow only makes
the KKT quantities of Section 2's termination tests infinite or NaN, which the check
turns into PDLP_NUMERICAL."""
import numpy as np
import pytest

import lpgen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pk():
    from paper_2312_14832_b300 import build
    build.build()
    import paper_2312_14832_b300 as pk
    return pk


def test_time_limit_returns_a_checked_point(pk):
    """A limit of 1 us ends the solve at the first check interval the host reads after it:
    TIME_LIMIT, a finite point, and relative errors that are the oracle's evaluation of
    that point on the unscaled LP."""
    lp = lpgen.planted_zipf(seed=4, n=200000, m=100000, nnz=2000000)
    with pk.Solver.from_lp(lp, scaling=1) as s:
        r = s.solve(tol=1e-10, time_limit_s=1e-6)
    assert r["status"] == pk.TIME_LIMIT
    assert 0 < r["iters"] < 100_000 and r["iters"] % 64 == 0
    assert np.all(np.isfinite(r["x"])) and np.all(np.isfinite(r["y"]))
    rp, rd, rg = oracle.relative_errors(lp, r["x"], r["y"])
    for got, want in ((r["rel_primal"], rp), (r["rel_dual"], rd), (r["rel_gap"], rg)):
        assert abs(got - want) <= 1e-8 * want + 1e-12
    assert max(rp, rd, rg) > 1e-10


def test_time_limit_not_reached(pk):
    """A generous limit changes nothing: the same iterations and status as without it."""
    lp = lpgen.planted_small(2)
    with pk.Solver.from_lp(lp) as s:
        a = s.solve(tol=1e-6, engine=1)
        b = s.solve(tol=1e-6, time_limit_s=600.0)
    assert a["status"] == b["status"] == pk.OPTIMAL and a["iters"] == b["iters"]


@pytest.mark.parametrize("engine", [1, 2])
def test_overflowing_step_is_numerical(pk, engine):
    """eta = 1e300 sends the free columns and then the duals to +-inf in the first steps;
    the first check sees a non-finite KKT and stops with NUMERICAL (both engines)."""
    lp = lpgen.planted_small(0)
    with pk.Solver.from_lp(lp, eta=1e300) as s:
        r = s.solve(tol=1e-4, max_iter=10_000, engine=engine)
        assert r["status"] == pk.NUMERICAL
        assert r["iters"] == 64
        # the handle stays usable: the same LP with the computed step size solves
    with pk.Solver.from_lp(lp) as s:
        assert s.solve(tol=1e-4, engine=engine)["status"] == pk.OPTIMAL


def test_batch_overflow_is_numerical_per_lp(pk):
    """In a batch every LP decides for itself: all overflow with eta = 1e300."""
    lps = lpgen.batch_planted(4, seed=3, n_lo=100, n_hi=400)
    with pk.BatchSolver.from_lps(lps, eta=1e300) as b:
        res = b.solve(tol=1e-4, max_iter=10_000)
    assert all(r["status"] == pk.NUMERICAL and r["iters"] == 64 for r in res)

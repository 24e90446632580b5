"""Mixed precision (params.precision = MIXED): FP32 iterations, FP64 checks and FP64
refinement.  The FP32 phase follows a different trajectory from the FP64 oracle, so
results are compared on what the method guarantees: the returned point passes the three
relative tests of Section 2 (re-evaluated here by the oracle's KKT routine on the
unscaled LP), and its objective agrees with the FP64 oracle's within the accuracy both
solutions are asked for (1e-3 relative at tol 1e-4; 1e-6 at tol 1e-8, as for FP64)."""
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


def check_point(lp, x, y, tol):
    rp, rd, rg = oracle.relative_errors(lp, x, y)
    slack = 1.0 + 1e-6   # unscaling of the returned point rounds
    assert rp <= tol * slack and rd <= tol * slack and rg <= tol * slack, (rp, rd, rg)


@pytest.mark.parametrize("scaling", [0, 1])
def test_mixed_mcf_at_1e4(pk, scaling):
    lp = lpgen.mcf(0, nodes=2000, arcs=10000)
    ref = oracle.solve(lp, tol=1e-4, scaling=scaling)
    with pk.Solver.from_lp(lp, scaling=scaling, precision=pk.MIXED) as s:
        r = s.solve(tol=1e-4)
    assert r["status"] == pk.OPTIMAL
    assert r["fp32_iters"] > 0
    check_point(lp, r["x"], r["y"], 1e-4)
    assert abs(r["primal_obj"] - ref["primal_obj"]) <= 1e-3 * abs(ref["primal_obj"])


@pytest.mark.parametrize("scaling", [0, 1])
def test_mixed_refines_to_1e8(pk, scaling):
    lp = lpgen.planted_small(2)
    ref = oracle.solve(lp, tol=1e-8, scaling=scaling)
    with pk.Solver.from_lp(lp, scaling=scaling, precision=pk.MIXED) as s:
        r = s.solve(tol=1e-8)
    assert r["status"] == pk.OPTIMAL
    assert 0 < r["fp32_iters"] < r["iters"]          # an FP32 phase, then FP64 refinement
    check_point(lp, r["x"], r["y"], 1e-8)
    assert abs(r["primal_obj"] - ref["primal_obj"]) <= 1e-6 * abs(ref["primal_obj"])
    assert abs(r["primal_obj"] - lp["obj_star"]) <= 1e-6 * abs(lp["obj_star"])


def test_mixed_mcf_refines_to_1e8(pk):
    """The multicommodity-flow family (+-1 incidence entries, capacity rows) at a size the
    oracle solves to 1e-8 in seconds: an FP32 phase, then the switch to FP64 and the
    refinement; the point passes the three tests at 1e-8 by the oracle's evaluation and
    the objective matches the FP64 oracle's solve to 1e-6."""
    lp = lpgen.mcf(0, nodes=500, arcs=2500)
    ref = oracle.solve(lp, tol=1e-8, scaling=1)
    assert ref["status"] == oracle.STATUS_OPTIMAL
    with pk.Solver.from_lp(lp, scaling=1, precision=pk.MIXED) as s:
        r = s.solve(tol=1e-8)
    assert r["status"] == pk.OPTIMAL
    assert 0 < r["fp32_iters"] < r["iters"]
    check_point(lp, r["x"], r["y"], 1e-8)
    assert abs(r["primal_obj"] - ref["primal_obj"]) <= 1e-6 * abs(ref["primal_obj"])


def test_mixed_loose_tolerance_stays_fp32(pk):
    lp = lpgen.planted_small(1)
    with pk.Solver.from_lp(lp, precision=pk.MIXED) as s:
        r = s.solve(tol=1e-3)
        assert r["status"] == pk.OPTIMAL
        assert r["fp32_iters"] == r["iters"]
        check_point(lp, r["x"], r["y"], 1e-3)
        mp, md = s.time_iterations(10)
        assert mp > 0 and md > 0


def test_mixed_iteration_limit(pk):
    lp = lpgen.planted_small(0)
    with pk.Solver.from_lp(lp, precision=pk.MIXED) as s:
        r = s.solve(tol=0.0, max_iter=300)
    assert r["iters"] == 300 and r["status"] == pk.ITER_LIMIT
    assert np.all(np.isfinite(r["x"])) and np.all(np.isfinite(r["y"]))

"""Checkpoint and resume of a single-LP solve (pdlp_get_state / pdlp_solve_resume; no
counterpart in the paper).  A solve stopped at an iteration limit on the check grid and
resumed to a larger limit must give the uninterrupted solve's iterates, restart list and
per-check records bit for bit, on the same handle and on a fresh handle loaded from the
saved bytes; the uninterrupted solve is itself held to the oracle.  Errors are made on the
host (wrong sizes, unsupported handles)."""
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


def _same(a, b):
    for key in ("status", "iters", "restarts", "which", "omega", "eta", "primal_obj", "dual_obj",
                "rel_primal", "rel_dual", "rel_gap", "accepted"):
        assert a[key] == b[key], key
    np.testing.assert_array_equal(a["x"], b["x"])
    np.testing.assert_array_equal(a["y"], b["y"])


@pytest.mark.parametrize("step_rule", [0, 1])
@pytest.mark.parametrize("split", [448, 512])
def test_resume_equals_uninterrupted_solve(pk, step_rule, split):
    """Split at 448 iterations, where the uninterrupted solve restarts (the repeated check
    must restart as the ordinary one did), and at 512, where it does not."""
    lp = lpgen.planted_small(3)
    kw = dict(scaling=1, engine=1, step_rule=step_rule)
    with pk.Solver.from_lp(lp, **kw) as a:
        full = a.solve(tol=0.0, max_iter=1024)
        full_restarts = a.restarts()
        full_cur = a.iterate(0)
        full_anchor = a.iterate(2)
        full_log = a.log()
    assert full["iters"] == 1024 and len(full_restarts) > 0
    assert (448 in full_restarts) and (512 not in full_restarts)
    ref = oracle.solve(lp, tol=0.0, max_iter=1024, scaling=1, step_rule=step_rule)
    np.testing.assert_array_equal(full_restarts, ref["restart_iters"])
    if step_rule == 0:
        assert np.abs(full["x"] - ref["x"]).max() <= 1e-10 * np.abs(ref["x"]).max()
    with pk.Solver.from_lp(lp, **kw) as b:
        half = b.solve(tol=0.0, max_iter=split)
        assert half["iters"] == split and half["status"] == pk.ITER_LIMIT
        state = b.get_state()
        again = b.resume(tol=0.0, max_iter=1024)
        _same(again, full)
        np.testing.assert_array_equal(b.restarts(), full_restarts)
        for got, want in zip(b.iterate(0), full_cur):
            np.testing.assert_array_equal(got, want)
        for got, want in zip(b.iterate(2), full_anchor):
            np.testing.assert_array_equal(got, want)
        assert b.log() == full_log
    with pk.Solver.from_lp(lp, **kw) as c:   # a fresh handle, loaded from the bytes
        loaded = c.resume(state=state, tol=0.0, max_iter=1024)
        _same(loaded, full)
        np.testing.assert_array_equal(c.restarts(), full_restarts)
        assert c.log() == full_log


def test_resume_to_tolerance(pk):
    """Stopped at 512 iterations on the way to 1e-7 and resumed: the same termination,
    iteration count and point as the uninterrupted solve."""
    lp = lpgen.planted_small(5)
    with pk.Solver.from_lp(lp, scaling=1, engine=1) as a:
        full = a.solve(tol=1e-7)
    assert full["status"] == pk.OPTIMAL and full["iters"] > 512
    with pk.Solver.from_lp(lp, scaling=1, engine=1) as b:
        b.solve(tol=1e-7, max_iter=512)
        again = b.resume(tol=1e-7, max_iter=100_000_000)
    _same(again, full)


def test_resume_errors(pk):
    lp = lpgen.planted_small(1)
    with pk.Solver.from_lp(lp, engine=1) as s:
        with pytest.raises(pk.SolverError):
            s.get_state()                      # nothing solved yet
        s.solve(tol=0.0, max_iter=128)
        state = s.get_state()
        with pytest.raises(pk.SolverError) as e:
            s.resume(state=state[:-8], max_iter=256)
        assert e.value.code == -1
        with pytest.raises(pk.SolverError):
            s.resume(state=b"x" * len(state), max_iter=256)
        with pytest.raises(pk.SolverError):
            s.resume(max_iter=256, engine=2)
    with pk.Solver.from_lp(lpgen.mcf(0, nodes=200, arcs=1000), engine=1) as other:
        with pytest.raises(pk.SolverError) as e:
            other.resume(state=state, max_iter=256)
        assert "other sizes" in str(e.value) or e.value.code == -1
    with pk.Solver.from_lp(lp, precision=pk.MIXED) as m:
        m.solve(tol=0.0, max_iter=128)
        with pytest.raises(pk.SolverError):
            m.get_state()
    with pk.Solver.from_lp(lp) as p:              # engine 0: the persistent engine
        p.solve(tol=0.0, max_iter=128)
        if p.info()["batch_team"] > 0:
            with pytest.raises(pk.SolverError):
                p.get_state()

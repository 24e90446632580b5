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


def _solve_mixed(pk, lp, scaling, values, **kw):
    with pk.Solver.from_lp(lp, scaling=scaling, precision=pk.MIXED, mixed_values=values) as s:
        r = s.solve(**kw)
        info = s.info()
    return r, info


@pytest.mark.parametrize("scaling", [0, 1])
def test_sign_bit_products_follow_the_fp64_oracle(pk, scaling):
    """K with +-1 entries stored as sign bits (mixed_values 0 picks it for the MCF LP, 2
    forces it): 192 FP32 iterations (three check intervals, tolerance 0) stay within the
    FP32 rounding of the FP64 oracle's iterates, element by element, like the FP32 value
    copies do.  A wrong sign, a scale applied twice or a padding slot that gathers a
    nonzero entry would move the iterates by O(1)."""
    lp = lpgen.mcf(1, nodes=500, arcs=2500)
    ref = oracle.solve(lp, tol=0.0, max_iter=192, scaling=scaling)
    got = {}
    for values in (0, 1, 2):
        r, info = _solve_mixed(pk, lp, scaling, values, tol=0.0, max_iter=192)
        assert info["mixed_values"] == (1 if values == 1 else 2)
        assert r["iters"] == 192 and r["fp32_iters"] == 192
        assert r["restarts"] == ref["restarts"]
        got[values] = r
        for key in ("x", "y"):
            want = ref[key]
            err = np.max(np.abs(r[key] - want)) / max(1.0, np.max(np.abs(want)))
            assert err <= 1e-4, (values, key, err)
    # automatic and forced sign bits run the same kernels on the same data: identical
    assert np.array_equal(got[0]["x"], got[2]["x"]) and np.array_equal(got[0]["y"], got[2]["y"])


def test_sign_bits_only_for_unit_entries(pk):
    """An LP with entries other than +-1 keeps FP32 value copies under automatic choice
    and is refused when sign bits are forced; FP64 handles report no FP32 products."""
    lp = lpgen.planted_small(0)
    with pk.Solver.from_lp(lp, precision=pk.MIXED) as s:
        assert s.info()["mixed_values"] == 1
    with pytest.raises(pk.SolverError) as e:
        pk.Solver.from_lp(lp, precision=pk.MIXED, mixed_values=2)
    assert e.value.code == -1 and "+1 or -1" in str(e.value)
    with pk.Solver.from_lp(lpgen.mcf(0, nodes=200, arcs=1000)) as s:
        assert s.info()["mixed_values"] == 0


@pytest.mark.parametrize("values", [1, 2])
def test_mcf_to_1e4_with_either_storage(pk, values):
    """Both storages of the FP32 products solve the MCF LP to 1e-4 (oracle's evaluation)
    with objectives within 1e-3 of the FP64 oracle's."""
    lp = lpgen.mcf(2, nodes=2000, arcs=10000)
    ref = oracle.solve(lp, tol=1e-4, scaling=1)
    r, info = _solve_mixed(pk, lp, 1, values, tol=1e-4)
    assert info["mixed_values"] == values
    assert r["status"] == pk.OPTIMAL and r["fp32_iters"] == r["iters"]
    check_point(lp, r["x"], r["y"], 1e-4)
    assert abs(r["primal_obj"] - ref["primal_obj"]) <= 1e-3 * abs(ref["primal_obj"])


def test_sign_bits_box_only(pk):
    """An LP with no rows has no entry other than +-1: sign bits are chosen, and the FP32
    iterations solve the box LP like the oracle."""
    lp = lpgen.box_only(3, n=100, free_frac=0.2)
    ref = oracle.solve(lp, tol=1e-6, max_iter=100000)
    with pk.Solver.from_lp(lp, precision=pk.MIXED) as s:
        assert s.info()["mixed_values"] == 2
        r = s.solve(tol=1e-6, max_iter=100000)
    assert r["status"] == pk.OPTIMAL
    err = np.max(np.abs(r["x"] - ref["x"])) / max(1.0, np.max(np.abs(ref["x"])))
    assert err <= 1e-5


def test_sign_bits_with_explicit_zero_entries(pk):
    """Explicit zero entries (stored pairs with value 0) leave the LP unchanged and still
    qualify for sign bits: a padding-like slot that gathers a zero.  The MCF LP with 500
    such entries added solves to 1e-4 by the oracle's evaluation, objective within 1e-3
    of the oracle's solve of the same stored LP."""
    base = lpgen.mcf(3, nodes=1000, arcs=5000)
    m, n = base["m"], base["n"]
    rp, ci, v = base["row_ptr"], base["col_idx"], base["val"]
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(rp))
    rng = np.random.default_rng(0)
    zr, zc = rng.integers(0, m, 500), rng.integers(0, n, 500)
    present = set(zip(rows.tolist(), ci.tolist()))
    keep = np.array([(a, b) not in present for a, b in zip(zr.tolist(), zc.tolist())])
    zr, zc = zr[keep], zc[keep]
    lp = dict(base)
    lp["row_ptr"], lp["col_idx"], lp["val"] = lpgen.csr_from_coo(
        m, n, np.concatenate([rows, zr]), np.concatenate([ci.astype(np.int64), zc]),
        np.concatenate([v, np.zeros(zr.shape[0])]))
    assert lp["row_ptr"][-1] == rp[-1] + zr.shape[0] and np.count_nonzero(lp["val"] == 0.0) == zr.shape[0]
    ref = oracle.solve(lp, tol=1e-4, scaling=1)
    r, info = _solve_mixed(pk, lp, 1, 0, tol=1e-4)
    assert info["mixed_values"] == 2
    assert r["status"] == pk.OPTIMAL
    check_point(lp, r["x"], r["y"], 1e-4)
    assert abs(r["primal_obj"] - ref["primal_obj"]) <= 1e-3 * abs(ref["primal_obj"])

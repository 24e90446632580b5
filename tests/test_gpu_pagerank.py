"""PageRank-shaped LPs (a dense equality row sum x = 1 over n columns, n sparse
inequality rows): the dense row is stored as a wide row (spread over the 32 lanes of a
chunk of its own).  Parity with the oracle as for every LP: SpMV rows within
1e-13 * sum |K_ij x_j|, the point after 1000 iterations within relative 1e-10, and the
solution at 1e-8 close to the PageRank vector.  With scaling these LPs reach machine
precision within 1000 iterations, where the choice between the current point and the
average is a tie, so the scaled cases stop at 200 iterations (errors near 1e-8)."""
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


def close_rel(a, b, rel):
    a, b = np.asarray(a), np.asarray(b)
    assert np.abs(a - b).max() <= rel * max(np.abs(b).max(), 1e-300)


# n = 2000: the dense row takes 63 slots (one warp task); n = 5000: 157 slots, split
# into pieces combined in order; the second dense row sits in the inequality block
CASES = [(2000, False), (5000, False), (3000, True)]


@pytest.mark.parametrize("n,extra", CASES)
def test_pagerank_spmv_with_wide_rows(pk, n, extra):
    lp = lpgen.pagerank(n, seed=2, dense_ineq_row=extra)
    K = sp.csr_matrix((lp["val"], lp["col_idx"], lp["row_ptr"]), shape=(lp["m"], lp["n"]))
    rng = np.random.default_rng(0)
    x = rng.standard_normal(lp["n"])
    y = rng.standard_normal(lp["m"])
    with pk.Solver.from_lp(lp) as s:
        assert s.info()["wide_rows_K"] == (2 if extra else 1)
        got = s.spmv(x)
        gott = s.spmv(y, transpose=True)
    assert np.all(np.abs(got - oracle.spmv(lp, x)) <= 1e-13 * (abs(K) @ np.abs(x)) + 1e-300)
    assert np.all(np.abs(gott - K.T @ y) <= 1e-13 * (abs(K).T @ np.abs(y)) + 1e-300)


@pytest.mark.parametrize("n,extra", CASES)
@pytest.mark.parametrize("scaling", [0, 1])
def test_pagerank_iterates_after_1000(pk, n, extra, scaling):
    lp = lpgen.pagerank(n, seed=3, dense_ineq_row=extra)
    iters = 200 if scaling else 1000
    ref = oracle.solve(lp, tol=0.0, max_iter=iters, scaling=scaling)
    with pk.Solver.from_lp(lp, scaling=scaling) as s:
        r = s.solve(tol=0.0, max_iter=iters)
    assert r["iters"] == iters and r["restarts"] == ref["restarts"] and r["which"] == ref["which"]
    assert abs(r["eta"] - ref["eta"]) <= 1e-12 * ref["eta"]
    close_rel(r["x"], ref["x"], 1e-10)
    close_rel(r["y"], ref["y"], 1e-10)


@pytest.mark.parametrize("step_rule", [0, 1])
def test_pagerank_solution_is_the_pagerank_vector(pk, step_rule):
    lp = lpgen.pagerank(5000, seed=4)
    with pk.Solver.from_lp(lp, scaling=1, step_rule=step_rule) as s:
        r = s.solve(tol=1e-8)
    assert r["status"] == pk.OPTIMAL
    xs = lp["x_star"]
    assert np.abs(r["x"] - xs).max() <= 1e-5 * xs.max()
    assert abs(r["x"].sum() - 1.0) <= 1e-7


def test_pagerank_mixed_precision(pk):
    lp = lpgen.pagerank(5000, seed=5)
    with pk.Solver.from_lp(lp, scaling=1, precision=pk.MIXED) as s:
        r = s.solve(tol=1e-6)
    assert r["status"] == pk.OPTIMAL and r["fp32_iters"] > 0
    rp, rd, rg = oracle.relative_errors(lp, r["x"], r["y"])
    assert max(rp, rd, rg) <= 1e-6 * (1 + 1e-6)

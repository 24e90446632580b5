"""Parity at the full size of the large workload: lpgen.planted_zipf(seed 0), n = 2e6,
m = 1e6, about 2e7 nonzeros, the LP bench.py times, set up as bench.py does (Ruiz +
Pock-Chambolle scaling, SpMV schedule chosen by the setup autotuner, the kernels
launched per iteration as CUDA graphs).

  * K x and K'y on sampled rows and columns (random ones, the longest, the ragged ends)
    against the oracle's SpMV of the sampled sub-matrices: 1e-12 of sum |K_ij v_j|
    (the products of the scaled layout carry a few extra roundings).
  * Two check intervals, 128 PDHG iterations, with their restart decisions: every
    element of the current and average iterates against the oracle at 1e-10 relative,
    the same restarts and primal weight.  eta is given (0.9, the step of this scaled LP
    to within 0.2 %), so the oracle skips its 100 power iterations on this LP.  The
    adaptive step rule likewise over 64 attempts.
  * The device layout builder against the host builder: bit-identical products (with
    one fixed schedule on both), so the radix sort and the fill hold at 2e7 entries.

The other full-size workloads, each in the configuration bench.py times:
  * the multicommodity-flow LP (n = 8e6, 2.4e7 nonzeros): one check interval in FP64
    element by element against the oracle (1e-10), and in FP32 with the +-1 entries as
    sign bits and as value copies (1e-4); MIXED (FP32 iterations, FP64 checks) to 1e-4,
    the returned point re-checked by the oracle's KKT routine, the objective within 1e-6
    of the FP64 solve;
  * the 4096-LP batch (5.5e8 nonzeros): the FP64 two-stage solve and the MIXED solve to
    1e-4; sampled LPs (evenly spaced, the largest, the one that reaches the iteration
    cap) solved by the oracle: the same status and iteration count and the objective
    within 1e-6 (FP64), the point within the tolerance and the objective within 1e-3
    (MIXED);
  * the 200 x 300 transportation family (n = 60000): eight members batched, cold and
    warm-started from a perturbed optimum, against the oracle from the same points.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import lpgen
import oracle

pytestmark = pytest.mark.gpu

ETA = 0.9


@pytest.fixture(scope="module")
def pk():
    from paper_2312_14832_b300 import build
    build.build()
    import paper_2312_14832_b300 as pk
    return pk


@pytest.fixture(scope="module")
def big():
    lp = lpgen.planted_zipf(seed=0)
    K = sp.csr_matrix((lp["val"], lp["col_idx"], lp["row_ptr"]), shape=(lp["m"], lp["n"]))
    return lp, K


def _sample(rng, lengths, count):
    order = np.argsort(-lengths, kind="stable")
    n = lengths.shape[0]
    pick = np.concatenate([rng.choice(n, count, replace=False), order[:50], order[-50:],
                           np.arange(max(0, n - 40), n)])
    return np.unique(pick)


def _rows_lp(M, rows):
    S = M[rows].tocsr()
    return dict(m=S.shape[0], n=S.shape[1], row_ptr=S.indptr.astype(np.int64), col_idx=S.indices.astype(np.int32),
                val=S.data)


def test_fullsize_spmv_on_sampled_rows_and_columns(pk, big):
    lp, K = big
    rng = np.random.default_rng(1)
    x = rng.standard_normal(lp["n"])
    y = rng.standard_normal(lp["m"])
    rows = _sample(rng, np.diff(K.indptr), 2000)
    Kt = K.T.tocsr()
    cols = _sample(rng, np.diff(Kt.indptr), 2000)
    with pk.Solver.from_lp(lp, scaling=1) as s:
        assert s.info()["tasks_K"] > 10000   # the autotuned schedule of the full LP
        kx = s.spmv(x)
        kty = s.spmv(y, transpose=True)
    A = abs(K)
    want = oracle.spmv(_rows_lp(K, rows), x)
    assert np.all(np.abs(kx[rows] - want) <= 1e-12 * (A[rows] @ np.abs(x)) + 1e-300)
    want_t = oracle.spmv(_rows_lp(Kt, cols), y)
    assert np.all(np.abs(kty[cols] - want_t) <= 1e-12 * (A.T.tocsr()[cols] @ np.abs(y)) + 1e-300)


@pytest.mark.parametrize("step_rule,iters", [(0, 128), (1, 64)])
def test_fullsize_check_intervals(pk, big, step_rule, iters):
    lp, _ = big
    ref = oracle.solve(lp, tol=0.0, max_iter=iters, scaling=1, eta=ETA, step_rule=step_rule)
    with pk.Solver.from_lp(lp, scaling=1, eta=ETA, step_rule=step_rule) as s:
        r = s.solve(tol=0.0, max_iter=iters)
        assert r["launches"] > 1   # the kernels launched per iteration, as in the bench
        assert r["iters"] == ref["iters"] == iters
        np.testing.assert_array_equal(s.restarts(), ref["restart_iters"])
        xc, yc = s.iterate(0)
        xa, ya = s.iterate(1)
    for got, want in ((xc, ref["x_cur"]), (yc, ref["y_cur"]), (xa, ref["x_avg"]), (ya, ref["y_avg"])):
        scale = np.abs(want).max()
        assert np.abs(got - want).max() <= 1e-10 * scale
        assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)
    assert abs(r["omega"] - ref["omega"]) <= 1e-10 * ref["omega"]


def test_fullsize_device_builder_equals_host_builder(pk, big):
    lp, _ = big
    fixed = dict(tile_slots=32, tile_chunks=4, spmv_batch=8)
    rng = np.random.default_rng(3)
    x, y = rng.standard_normal(lp["n"]), rng.standard_normal(lp["m"])
    with pk.Solver.from_lp(lp, scaling=1, **fixed) as a:
        ax, ay = a.spmv(x), a.spmv(y, transpose=True)
    with pk.Solver.from_lp(lp, scaling=1, host_layout=1, **fixed) as b:
        np.testing.assert_array_equal(ax, b.spmv(x))
        np.testing.assert_array_equal(ay, b.spmv(y, transpose=True))


def _check_point(lp, x, y, tol):
    rp, rd, rg = oracle.relative_errors(lp, x, y)
    assert max(rp, rd, rg) <= tol * (1 + 1e-6), (rp, rd, rg)


def test_fullsize_mcf(pk):
    lp = lpgen.mcf(0)
    iters = 64
    ref = oracle.solve(lp, tol=0.0, max_iter=iters, scaling=1, eta=ETA)
    with pk.Solver.from_lp(lp, scaling=1, eta=ETA) as s:
        r = s.solve(tol=0.0, max_iter=iters)
        assert r["iters"] == ref["iters"] == iters
        np.testing.assert_array_equal(s.restarts(), ref["restart_iters"])
        xc, yc = s.iterate(0)
    for got, want in ((xc, ref["x_cur"]), (yc, ref["y_cur"])):
        assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
    # the FP32 iterations over the same interval, with the +-1 entries as sign bits (the
    # automatic choice here) and as FP32 value copies: within FP32 rounding of the oracle
    for values, storage in ((0, 2), (1, 1)):
        with pk.Solver.from_lp(lp, scaling=1, eta=ETA, precision=pk.MIXED, mixed_values=values) as s:
            assert s.info()["mixed_values"] == storage
            r = s.solve(tol=0.0, max_iter=iters, mixed_switch_tol=1e-30)
            assert r["fp32_iters"] == iters
            xc, yc = s.iterate(0)
        for got, want in ((xc, ref["x_cur"]), (yc, ref["y_cur"])):
            assert np.abs(got - want).max() <= 1e-4 * np.abs(want).max(), (storage, np.abs(got - want).max())
    with pk.Solver.from_lp(lp, scaling=1) as s:
        r64 = s.solve(tol=1e-4)
    with pk.Solver.from_lp(lp, scaling=1, precision=pk.MIXED) as s:
        rm = s.solve(tol=1e-4)
    assert r64["status"] == rm["status"] == pk.OPTIMAL
    assert rm["fp32_iters"] > 0
    _check_point(lp, r64["x"], r64["y"], 1e-4)
    _check_point(lp, rm["x"], rm["y"], 1e-4)
    assert abs(rm["primal_obj"] - r64["primal_obj"]) <= 1e-6 * abs(r64["primal_obj"])


def test_fullsize_batch_4096(pk):
    lps = lpgen.batch_planted(4096, seed=0)
    nnz = np.array([lp["val"].shape[0] for lp in lps])
    with pk.BatchSolver.from_lps(lps) as b:
        res = b.solve(tol=1e-4, max_iter=200000, want_points=False, batch_tail_iters=8192)
    its = np.array([r["iters"] for r in res])
    sample = sorted(set(range(0, 4096, 512)) | {int(np.argmax(nnz)), int(np.argmax(its))})
    with pk.BatchSolver.from_lps([lps[i] for i in sample]) as b:   # the sampled LPs' points
        pts = b.solve(tol=1e-4, max_iter=200000)
    with pk.BatchSolver.from_lps(lps, precision=pk.MIXED) as b:
        rm = b.solve(tol=1e-4, max_iter=200000, want_points=False)
    del b
    for k, i in enumerate(sample):
        lp, r = lps[i], res[i]
        ref = oracle.solve(lp, tol=1e-4, max_iter=200000)
        assert r["status"] == ref["status"], i
        assert r["iters"] == ref["iters"] == pts[k]["iters"], i
        if ref["status"] == pk.OPTIMAL:
            assert abs(r["primal_obj"] - ref["primal_obj"]) <= 1e-6 * (1 + abs(ref["primal_obj"])), i
            _check_point(lp, pts[k]["x"], pts[k]["y"], 1e-4)
            assert rm[i]["status"] == pk.OPTIMAL, i
            assert abs(rm[i]["primal_obj"] - ref["primal_obj"]) <= 1e-3 * (1 + abs(ref["primal_obj"])), i
        else:
            close = np.abs(pts[k]["x"] - ref["x"]).max() <= 1e-8 * max(np.abs(ref["x"]).max(), 1.0)
            assert close, i


def test_fullsize_transport_family_cold_and_warm(pk):
    fam = lpgen.transport_family(200, 300, seed=0)
    lps = [lpgen.transport_instance(fam, s) for s in range(100001, 100009)]
    refs = [oracle.solve(lp, tol=1e-4) for lp in lps]
    rng = np.random.default_rng(5)
    x0 = [np.maximum(r["x"] * (1 + 0.05 * rng.standard_normal(lp["n"])), 0.0) for lp, r in zip(lps, refs)]
    y0 = [r["y"] * (1 + 0.05 * rng.standard_normal(lp["m"])) for lp, r in zip(lps, refs)]
    w0 = [1.0] * len(lps)
    with pk.BatchSolver.from_lps(lps) as b:
        cold = b.solve(tol=1e-4)
        warm = b.solve(tol=1e-4, x0=x0, y0=y0, omega0=w0)
        assert b.info()["batch_resident"] == 3   # iterates in global memory, as in the bench
    for i, lp in enumerate(lps):
        wref = oracle.solve(lp, tol=1e-4, x0=x0[i], y0=y0[i], omega0=w0[i])
        for r, ref in ((cold[i], refs[i]), (warm[i], wref)):
            assert r["status"] == ref["status"] == pk.OPTIMAL
            assert r["iters"] == ref["iters"]
            assert abs(r["primal_obj"] - ref["primal_obj"]) <= 1e-6 * (1 + abs(ref["primal_obj"]))
            _check_point(lp, r["x"], r["y"], 1e-4)

"""The device layout builder (default) against the host builder (host_layout=1).

Both must produce the same SELL-32 layouts of K and K' (rows by decreasing length,
equality rows first, wide rows spread over a chunk; K rows in the caller's entry order,
K' rows by increasing row; padding columns inside each LP's range), so with the same
schedule parameters the products K v and K' v agree bit for bit: single-LP handles
built both ways, batches built both ways, and a single-LP handle against a batch
holding only that LP.  The cases span one to three radix passes of the CSC sort (n up
to 2^17), several scan tiles, ragged tails, empty rows, columns and LPs, repeated
columns within a row, equality rows and wide rows; scipy checks the products besides
(1e-13 of sum |K_ij v_j| per row).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import lpgen

pytestmark = pytest.mark.gpu

SCHEDULE = dict(tile_slots=64, tile_chunks=4, spmv_batch=8)


@pytest.fixture(scope="module")
def pk():
    from paper_2312_14832_b300 import build
    build.build()
    import paper_2312_14832_b300 as pk
    return pk


def _lp(seed, m, n, max_len, m1_frac=0.3, zipf=True, repeats=True):
    """Row lengths up to max_len (< 1024, so no wide rows); columns Zipf-skewed (long
    and empty columns), drawn with replacement when repeats (repeated columns in a row)."""
    rng = np.random.default_rng(seed)
    lengths = rng.integers(0, max_len + 1, size=m)
    lengths[rng.random(m) < 0.05] = 0
    rows = np.repeat(np.arange(m), lengths)
    if zipf:
        w = 1.0 / np.arange(1, n + 1) ** 1.1
        cols = rng.choice(n, size=rows.size, p=w / w.sum())
    else:
        cols = rng.integers(0, n, size=rows.size)
    if not repeats:
        keep = np.unique(rows.astype(np.int64) * n + cols, return_index=True)[1]
        keep.sort()
        rows, cols = rows[keep], cols[keep]
    vals = rng.standard_normal(rows.size) * 10.0 ** rng.uniform(-2, 2, rows.size)
    rp = np.zeros(m + 1, dtype=np.int64)
    np.add.at(rp, rows + 1, 1)
    rp = np.cumsum(rp)
    order = np.argsort(rows, kind="stable")   # already row-major; keeps in-row order
    return dict(m=m, n=n, m1=int(m * m1_frac), row_ptr=rp, col_idx=cols[order].astype(np.int32),
                val=vals[order], c=rng.standard_normal(n), q=rng.standard_normal(m),
                l=-np.ones(n), u=np.ones(n))


CASES = {
    "tiny": (0, 40, 30, 6),
    "two_passes": (1, 700, 300, 40),
    "three_passes": (2, 6000, 70000, 120),
    "tall": (3, 50000, 900, 25),
    "ragged": (4, 33, 100001, 700),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("scaling", [0, 1])
def test_device_layout_equals_host_layout(pk, case, scaling):
    seed, m, n, max_len = CASES[case]
    lp = _lp(seed, m, n, max_len)
    rng = np.random.default_rng(seed + 100)
    x = rng.standard_normal(n)
    y = rng.standard_normal(m)
    with pk.Solver.from_lp(lp, scaling=scaling, **SCHEDULE) as s, \
            pk.BatchSolver.from_lps([lp], scaling=scaling, **SCHEDULE) as b:
        assert s.info()["wide_rows_K"] == 0
        kx, kty = s.spmv(x), s.spmv(y, transpose=True)
        np.testing.assert_array_equal(kx, b.spmv(x))
        np.testing.assert_array_equal(kty, b.spmv(y, transpose=True))
    K = sp.csr_matrix((lp["val"], lp["col_idx"], lp["row_ptr"]), shape=(m, n))
    A = abs(K)
    assert np.all(np.abs(kx - K @ x) <= 1e-13 * (A @ np.abs(x)) + 1e-300)
    assert np.all(np.abs(kty - K.T @ y) <= 1e-13 * (A.T @ np.abs(y)) + 1e-300)


WIDE = {"wide_rows": (8, 3000, 5000, 30)}


@pytest.mark.parametrize("case", list(CASES) + list(WIDE))
def test_device_builder_equals_host_builder(pk, case):
    seed, m, n, max_len = {**CASES, **WIDE}[case]
    lp = _lp(seed, m, n, max_len)
    if case in WIDE:   # two dense rows (one equality, one inequality): wide rows
        rp, ci, v = lp["row_ptr"], lp["col_idx"], lp["val"]
        rows = [np.arange(n, dtype=np.int32)[::s] for s in (1, 2)]
        lens = np.diff(rp)
        lens[0], lens[-1] = rows[0].size, rows[1].size
        newc = [rows[0]] + [ci[rp[i]:rp[i + 1]] for i in range(1, m - 1)] + [rows[1]]
        lp = dict(lp, row_ptr=np.concatenate([[0], np.cumsum(lens)]).astype(np.int64),
                  col_idx=np.concatenate(newc).astype(np.int32),
                  val=np.random.default_rng(9).standard_normal(int(lens.sum())))
    rng = np.random.default_rng(seed + 200)
    x, y = rng.standard_normal(n), rng.standard_normal(m)
    with pk.Solver.from_lp(lp, scaling=1, **SCHEDULE) as a, \
            pk.Solver.from_lp(lp, scaling=1, host_layout=1, **SCHEDULE) as b:
        assert a.info()["wide_rows_K"] == b.info()["wide_rows_K"] == (2 if case in WIDE else 0)
        np.testing.assert_array_equal(a.spmv(x), b.spmv(x))
        np.testing.assert_array_equal(a.spmv(y, transpose=True), b.spmv(y, transpose=True))
        r1, r2 = a.solve(max_iter=300, tol=0.0), b.solve(max_iter=300, tol=0.0)
        np.testing.assert_array_equal(r1["x"], r2["x"])
        np.testing.assert_array_equal(r1["y"], r2["y"])


def test_batch_device_builder_equals_host_builder(pk):
    """A batch of varied LPs (an LP without rows, a one-column LP, ragged sizes): both
    builders give identical products and identical batched solves."""
    lps = [_lp(20 + i, m, n, L) for i, (m, n, L) in
           enumerate([(300, 500, 30), (0, 40, 1), (50, 1, 1), (1200, 900, 60), (33, 70001, 200), (7, 7, 7)])]
    M, N = sum(lp["m"] for lp in lps), sum(lp["n"] for lp in lps)
    rng = np.random.default_rng(30)
    x, y = rng.standard_normal(N), rng.standard_normal(M)
    with pk.BatchSolver.from_lps(lps, scaling=1, **SCHEDULE) as a, \
            pk.BatchSolver.from_lps(lps, scaling=1, host_layout=1, **SCHEDULE) as b:
        np.testing.assert_array_equal(a.spmv(x), b.spmv(x))
        np.testing.assert_array_equal(a.spmv(y, transpose=True), b.spmv(y, transpose=True))
        ra, rb = a.solve(max_iter=256, tol=0.0), b.solve(max_iter=256, tol=0.0)
        for u, v in zip(ra, rb):
            np.testing.assert_array_equal(u["x"], v["x"])
            np.testing.assert_array_equal(u["y"], v["y"])
    blocks = [sp.csr_matrix((lp["val"], lp["col_idx"], lp["row_ptr"]), shape=(lp["m"], lp["n"])) for lp in lps]
    K = sp.block_diag(blocks, format="csr")
    kx = K @ x
    with pk.BatchSolver.from_lps(lps, scaling=1) as a:
        assert np.all(np.abs(a.spmv(x) - kx) <= 1e-13 * (abs(K) @ np.abs(x)) + 1e-300)


def test_batch_column_outside_its_lp_is_rejected(pk):
    """A column index valid for the whole batch but not for its own LP is an error."""
    lps = [_lp(40, 100, 50, 10), _lp(41, 100, 80, 10)]
    bad = dict(lps[0], col_idx=lps[0]["col_idx"].copy())
    bad["col_idx"][5] = 60   # < 130 columns in total, >= 50 of LP 0
    with pytest.raises(pk.SolverError) as e:
        pk.BatchSolver.from_lps([bad, lps[1]])
    assert "column index" in str(e.value)


def test_device_inputs_give_the_same_layout(pk):
    """Device-resident inputs (copied device to device) build the same layout as host
    inputs: identical products."""
    import torch
    lp = _lp(5, 3000, 20000, 60)
    dev = {k: (torch.as_tensor(v).cuda() if isinstance(v, np.ndarray) else v) for k, v in lp.items()}
    x = np.random.default_rng(6).standard_normal(lp["n"])
    with pk.Solver.from_lp(lp, scaling=1, **SCHEDULE) as a, pk.Solver.from_lp(dev, scaling=1, **SCHEDULE) as b:
        np.testing.assert_array_equal(a.spmv(x), b.spmv(torch.as_tensor(x).cuda()).cpu().numpy())


def test_empty_matrix_and_no_rows(pk):
    """nnz = 0 (one row without entries) and m = 0: the layouts are padding only."""
    n = 50
    base = dict(n=n, c=np.ones(n), l=np.zeros(n), u=np.ones(n))
    for m in (0, 1):
        lp = dict(base, m=m, m1=0, row_ptr=np.zeros(m + 1, dtype=np.int64), col_idx=np.zeros(0, np.int32),
                  val=np.zeros(0), q=np.zeros(m))
        with pk.Solver.from_lp(lp, scaling=1) as s:
            assert np.all(s.spmv(np.ones(n)) == 0.0)
            if m:
                assert np.all(s.spmv(np.ones(m), transpose=True) == 0.0)
            r = s.solve(tol=1e-8)
            np.testing.assert_allclose(r["x"], np.zeros(n), atol=1e-8)


def test_invalid_entries_are_rejected_on_the_device(pk):
    """Column indices out of range (either side) and non-finite values are found by the
    device check; a non-finite value is reported first, as before."""
    lp = _lp(7, 200, 300, 20)
    for k, v in (("col_idx", -1), ("col_idx", 300), ("val", np.inf), ("val", np.nan)):
        bad = dict(lp, **{k: lp[k].copy()})
        bad[k][len(bad[k]) // 2] = v
        with pytest.raises(pk.SolverError) as e:
            pk.Solver.from_lp(bad)
        assert ("column index" in str(e.value)) == (k == "col_idx")


@pytest.mark.parametrize("host_layout", [0, 1])
def test_batch_setup_from_device_arrays(pk, host_layout):
    """pdlp_batch_setup with every array on the device (params.inputs_on_device = 1,
    called through the C ABI): the same products and the same batched solve as the
    same LPs from host arrays."""
    import ctypes as C
    import torch
    from paper_2312_14832_b300 import _lib
    lps = [_lp(50 + i, m, n, L) for i, (m, n, L) in enumerate([(300, 500, 30), (0, 40, 1), (1200, 900, 60)])]
    M, N = sum(lp["m"] for lp in lps), sum(lp["n"] for lp in lps)
    lib = _lib.load()
    sizes = [np.array([lp[k] for lp in lps], dtype=np.int64) for k in ("m", "n", "m1")]
    cat = lambda key, dt: torch.as_tensor(np.concatenate([np.asarray(lp[key], dtype=dt) for lp in lps])).cuda()
    dev = [cat("row_ptr", np.int64), cat("col_idx", np.int32), cat("val", np.float64), cat("c", np.float64),
           cat("q", np.float64), cat("l", np.float64), cat("u", np.float64)]
    torch.cuda.synchronize()
    p = pk.default_params(scaling=1, host_layout=host_layout, **SCHEDULE)
    p.inputs_on_device = 1
    h = C.c_void_p()
    rc = lib.pdlp_batch_setup(C.byref(h), len(lps), *[a.ctypes.data for a in sizes],
                              *[t.data_ptr() for t in dev], C.byref(p))
    assert rc == 0, lib.pdlp_last_error(None).decode()
    try:
        rng = np.random.default_rng(60)
        x, y = rng.standard_normal(N), rng.standard_normal(M)
        outs = []
        for v, tr, size in ((x, 0, M), (y, 1, N)):
            vin = torch.as_tensor(v).cuda()
            out = torch.empty(size, dtype=torch.float64, device="cuda")
            assert lib.pdlp_spmv(h, tr, vin.data_ptr(), out.data_ptr()) == 0
            outs.append(out.cpu().numpy())
        res = (_lib.Result * len(lps))()
        xo = torch.empty(N, dtype=torch.float64, device="cuda")
        yo = torch.empty(M, dtype=torch.float64, device="cuda")
        q = _lib.Params()
        C.memmove(C.byref(q), C.byref(p), C.sizeof(q))
        q.tol, q.max_iter = 0.0, 256
        assert lib.pdlp_batch_solve(h, C.byref(q), None, None, None, res, xo.data_ptr(), yo.data_ptr()) == 0
        xd, yd = xo.cpu().numpy(), yo.cpu().numpy()
    finally:
        lib.pdlp_free(h)
    with pk.BatchSolver.from_lps(lps, scaling=1, **SCHEDULE) as b:
        np.testing.assert_array_equal(outs[0], b.spmv(x))
        np.testing.assert_array_equal(outs[1], b.spmv(y, transpose=True))
        ref = b.solve(max_iter=256, tol=0.0)
    np.testing.assert_array_equal(xd, np.concatenate([r["x"] for r in ref]))
    np.testing.assert_array_equal(yd, np.concatenate([r["y"] for r in ref]))

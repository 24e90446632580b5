"""pdlp_spmv_csr_noalloc: the handle-less SpMV for callers that cannot allocate device
memory when they need K x (their device memory is all handed to their own allocator,
or they cannot afford cudaMalloc's implicit synchronisation).  It keeps its partial
sums in a fixed device array of the library instead of allocating.

Checked through the C ABI against the existing pdlp_spmv (a solver handle on the same
matrix, scaling off), on two calls in a row, within the SpMV tolerance of the other
GPU tests: |difference| <= 1e-13 * sum_j |K_ij x_j| per row.  This file is collected
last so that a run stopping at its first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import scipy.sparse as sp

import lpgen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_2312_14832_b300 import build
    build.build()
    import torch

    import paper_2312_14832_b300 as pk
    from paper_2312_14832_b300 import _lib
    return pk, _lib.load(), torch


def _call(lib, torch, m, n, rp, ci, v, x):
    d = lambda a, dt: torch.as_tensor(a, dtype=dt, device="cuda").contiguous()
    drp, dci, dv, dx = d(rp, torch.int64), d(ci, torch.int32), d(v, torch.float64), d(x, torch.float64)
    y = torch.full((m,), np.nan, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    rc = lib.pdlp_spmv_csr_noalloc(m, n, int(rp[-1]), drp.data_ptr(), dci.data_ptr(), dv.data_ptr(),
                                   dx.data_ptr(), y.data_ptr(), stream.cuda_stream)
    assert rc == 0, lib.pdlp_last_error(None)
    stream.synchronize()
    return y.cpu().numpy()


def test_noalloc_spmv_matches_pdlp_spmv_twice(env):
    pk, lib, torch = env
    # empty rows, short rows, rows crossing one and many 64-entry runs, a trailing empty row
    lengths = [0, 1, 63, 64, 65, 0, 5, 200, 1, 10000, 2, 130, 0] * 6 + [0]
    n = 15000
    rp, ci, v = lpgen.random_csr(21, len(lengths), n, lengths, dist="wide")
    m = len(lengths)
    lp = dict(m=m, n=n, m1=0, row_ptr=rp, col_idx=ci, val=v, c=np.zeros(n), q=np.zeros(m),
              l=np.full(n, -np.inf), u=np.full(n, np.inf))
    K = abs(sp.csr_matrix((v, ci, rp), shape=(m, n)))
    rng = np.random.default_rng(5)
    with pk.Solver.from_lp(lp) as s:
        for _ in range(2):   # two calls in a row share the scratch
            x = rng.standard_normal(n)
            want = s.spmv(x)
            got = _call(lib, torch, m, n, rp, ci, v, x)
            bound = 1e-13 * (K @ np.abs(x)) + 1e-300
            assert np.all(np.abs(got - want) <= bound)
            assert np.all(got[np.diff(rp) == 0] == 0.0)


def test_noalloc_spmv_allocates_nothing(env):
    """After a first call (which looks up the scratch address), further calls leave the
    device's free memory unchanged: an 8 MiB cudaMalloc would show in mem_get_info."""
    pk, lib, torch = env
    lengths = [3, 0, 200, 70, 1] * 40
    n = 5000
    rp, ci, v = lpgen.random_csr(8, len(lengths), n, lengths, dist="wide")
    m = len(lengths)
    d = lambda a, dt: torch.as_tensor(a, dtype=dt, device="cuda").contiguous()
    drp, dci, dv = d(rp, torch.int64), d(ci, torch.int32), d(v, torch.float64)
    dx = d(np.random.default_rng(2).standard_normal(n), torch.float64)
    y = torch.empty(m, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    call = lambda: lib.pdlp_spmv_csr_noalloc(m, n, int(rp[-1]), drp.data_ptr(), dci.data_ptr(), dv.data_ptr(),
                                             dx.data_ptr(), y.data_ptr(), stream.cuda_stream)
    assert call() == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        assert call() == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    # y == x is refused before any device work
    sq = lib.pdlp_spmv_csr_noalloc(n, n, int(rp[-1]), drp.data_ptr(), dci.data_ptr(), dv.data_ptr(),
                                   dx.data_ptr(), dx.data_ptr(), stream.cuda_stream)
    assert sq == -1 and b"overlap" in lib.pdlp_last_error(None)


def test_noalloc_spmv_empty_cases(env):
    """nnz = 0 (every row empty: no runs, only the fix-up kernel writes y, zeros) and
    m = 0 (nothing to do)."""
    pk, lib, torch = env
    m, n = 300, 40
    rp = np.zeros(m + 1, dtype=np.int64)
    got = _call(lib, torch, m, n, rp, np.zeros(0, dtype=np.int32), np.zeros(0), np.ones(n))
    assert np.all(got == 0.0)
    assert lib.pdlp_spmv_csr_noalloc(0, n, 0, None, None, None, None, None, None) == 0


def test_noalloc_spmv_rejects_sizes_beyond_the_scratch(env):
    pk, lib, torch = env
    rc = lib.pdlp_spmv_csr_noalloc(10, 10, 22_369_601, None, None, None, None, None, None)
    assert rc == -1
    assert b"scratch limit" in lib.pdlp_last_error(None)
    # the largest accepted size: 22,369,600 nonzeros in 1000 rows, against pdlp_spmv
    nnz = 22_369_600
    m, n = 1000, 2_000_000
    rng = np.random.default_rng(7)
    rp = np.linspace(0, nnz, m + 1).astype(np.int64)
    ci = rng.integers(0, n, nnz, dtype=np.int32)
    v = rng.standard_normal(nnz)
    x = rng.standard_normal(n)
    got = _call(lib, torch, m, n, rp, ci, v, x)
    lp = dict(m=m, n=n, m1=0, row_ptr=rp, col_idx=ci, val=v, c=np.zeros(n), q=np.zeros(m),
              l=np.full(n, -np.inf), u=np.full(n, np.inf))
    with pk.Solver.from_lp(lp) as s:
        want = s.spmv(x)
    K = abs(sp.csr_matrix((v, ci, rp), shape=(m, n)))
    assert np.all(np.abs(got - want) <= 1e-13 * (K @ np.abs(x)) + 1e-300)

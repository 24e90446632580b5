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


def test_noalloc_spmv_rejects_sizes_beyond_the_scratch(env):
    pk, lib, torch = env
    rc = lib.pdlp_spmv_csr_noalloc(10, 10, 22_369_601, None, None, None, None, None, None)
    assert rc == -1
    assert b"scratch limit" in lib.pdlp_last_error(None)

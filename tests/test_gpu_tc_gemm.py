"""The tcgen05 BF16 GEMM (pdlp_tc_gemm) against a float64 product of the same BF16
operands: |C - ref| <= 1e-5 * (|A| |B|^T) + 1e-30 elementwise (FP32 accumulation of
at most 1024 BF16 products, exact in FP32, rounding ~K * 2^-24 of the absolute sum)."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    from paper_2312_14832_b300 import build
    build.build()
    import torch
    from paper_2312_14832_b300 import _lib
    return _lib.load(), torch


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 384, 192), (128, 256, 1024), (384, 128, 128)])
@pytest.mark.parametrize("epi", ["plain", "bias_relu"])
def test_tc_gemm_matches_float64(env, M, N, K, epi):
    lib, torch = env
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    bias = torch.randn(N, generator=g).float() if epi == "bias_relu" else None
    dA, dB = A.cuda(), B.cuda()
    dbias = bias.cuda() if bias is not None else None
    out = torch.full((M, N), float("nan"), device="cuda")
    rc = lib.pdlp_tc_gemm(M, N, K, dA.data_ptr(), dB.data_ptr(), out.data_ptr(),
                          dbias.data_ptr() if dbias is not None else None, 1 if bias is not None else 0, None)
    assert rc == 0, lib.pdlp_last_error(None)
    a = A.double().numpy()
    b = B.double().numpy()
    ref = a @ b.T
    if bias is not None:
        ref = np.maximum(ref + bias.double().numpy()[None, :], 0.0)
    bound = 1e-5 * (np.abs(a) @ np.abs(b).T) + 1e-30
    got = out.cpu().double().numpy()
    assert np.all(np.abs(got - ref) <= bound + (1e-6 if bias is not None else 0.0))


def test_tc_gemm_rejects_bad_shapes(env):
    lib, torch = env
    assert lib.pdlp_tc_gemm(100, 128, 64, None, None, None, None, 0, None) == -1
    assert lib.pdlp_tc_gemm(128, 128, 48, None, None, None, None, 0, None) == -1

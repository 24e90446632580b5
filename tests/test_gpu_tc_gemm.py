"""The tcgen05 BF16 GEMM (pdlp_tc_gemm, pdlp_tc_gemm_split) against a float64 product of
the same BF16 operands: |C - ref| <= tol * (|A| |B|^T) + 1e-30 elementwise.  Each BF16
product is exact in FP32; the FP32 sums round by at most ~K * 2^-24 of the absolute sum
(tol = 1e-5 for K <= 1024, where the observed error is far below that bound, and
K * 2^-24 above)."""
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


def _operands(torch, M, N, K, seed):
    g = torch.Generator(device="cpu").manual_seed(seed)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    bias = torch.randn(N, generator=g).float()
    return A, B, bias


def _reference(A, B, bias, relu):
    a, b = A.double().numpy(), B.double().numpy()
    ref = a @ b.T + bias.double().numpy()[None, :]
    if relu:
        ref = np.maximum(ref, 0.0)
    return ref, np.abs(a) @ np.abs(b).T


@pytest.mark.parametrize("M,N,K", [(256, 256, 4096), (128, 384, 704)])
def test_tc_gemm_long_k(env, M, N, K):
    """K of 64 and 11 steps: the 6-stage ring is refilled many times."""
    lib, torch = env
    A, B, bias = _operands(torch, M, N, K, 11)
    out = torch.full((M, N), float("nan"), device="cuda")
    dA, dB, db = A.cuda(), B.cuda(), bias.cuda()   # kept alive across the call
    rc = lib.pdlp_tc_gemm(M, N, K, dA.data_ptr(), dB.data_ptr(), out.data_ptr(), db.data_ptr(), 0, None)
    assert rc == 0, lib.pdlp_last_error(None)
    ref, mag = _reference(A, B, bias, False)
    tol = max(1e-5, K * 2.0 ** -24)
    assert np.all(np.abs(out.cpu().double().numpy() - ref) <= tol * mag + 1e-6)


@pytest.mark.parametrize("splits", [1, 2, 5, 16, 40])
@pytest.mark.parametrize("relu", [0, 1])
def test_tc_gemm_split_k(env, splits, relu):
    """K cut into slices computed by separate CTAs and added in slice order (40 slices of
    a 1920-deep K become 30, one step each); bias and ReLU after the sum."""
    lib, torch = env
    M, N, K = 256, 128, 1920
    A, B, bias = _operands(torch, M, N, K, 5 + splits)
    ws = torch.empty(splits * M * N, device="cuda")
    out = torch.full((M, N), float("nan"), device="cuda")
    dA, dB, db = A.cuda(), B.cuda(), bias.cuda()
    rc = lib.pdlp_tc_gemm_split(M, N, K, dA.data_ptr(), dB.data_ptr(), out.data_ptr(), db.data_ptr(), relu, splits,
                                ws.data_ptr(), None)
    assert rc == 0, lib.pdlp_last_error(None)
    ref, mag = _reference(A, B, bias, relu)
    tol = K * 2.0 ** -24
    assert np.all(np.abs(out.cpu().double().numpy() - ref) <= tol * mag + 1e-6)


def test_tc_gemm_rejects_misaligned_operands(env):
    lib, torch = env
    A = torch.zeros(128 * 64 + 8, dtype=torch.bfloat16, device="cuda")
    B = torch.zeros(128 * 64, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(128 * 128, device="cuda")
    assert lib.pdlp_tc_gemm(128, 128, 64, A.data_ptr() + 2, B.data_ptr(), C.data_ptr(), None, 0, None) == -1
    assert lib.pdlp_tc_gemm_split(128, 128, 64, A.data_ptr(), B.data_ptr(), C.data_ptr(), None, 0, 2, None,
                                  None) == -1


def test_tc_gemm_rejects_bad_shapes(env):
    lib, torch = env
    assert lib.pdlp_tc_gemm(100, 128, 64, None, None, None, None, 0, None) == -1
    assert lib.pdlp_tc_gemm(128, 128, 48, None, None, None, None, 0, None) == -1


def test_bounded_wait_gives_up_and_context_stays_usable(env):
    """The MMA thread's first mbarrier wait with every operand copy withheld: it gives up
    after the poll limit, the call returns PDLP_ETIMEOUT (-4) without writing C, the kernel
    frees its tensor memory, and the next GEMM on the same context is correct."""
    lib, torch = env
    A, B, bias = _operands(torch, 128, 128, 64, seed=11)
    dA, dB = A.cuda(), B.cuda()
    out = torch.full((128, 128), -7.0, device="cuda")
    assert lib.pdlp_tc_gemm_wait_selftest(dA.data_ptr(), dB.data_ptr(), out.data_ptr(), 0, None) == -1
    rc = lib.pdlp_tc_gemm_wait_selftest(dA.data_ptr(), dB.data_ptr(), out.data_ptr(), 2000, None)
    assert rc == -4, lib.pdlp_last_error(None)
    assert b"gave up" in lib.pdlp_last_error(None)
    assert torch.all(out == -7.0)
    torch.cuda.synchronize()
    rc = lib.pdlp_tc_gemm(128, 128, 64, dA.data_ptr(), dB.data_ptr(), out.data_ptr(), None, 0, None)
    assert rc == 0, lib.pdlp_last_error(None)
    ref, scale = _reference(A, B, torch.zeros(128), False)
    assert np.all(np.abs(out.cpu().double().numpy() - ref) <= 1e-5 * scale + 1e-30)


@pytest.mark.parametrize("M,N,K,splits,relu", [(256, 18944, 128, 1, 1), (768, 384, 4096, 1, 0),
                                                (512, 256, 8192, 4, 1), (256, 1024, 4352, 17, 0)])
def test_tc_gemm_two_row_tiles(env, M, N, K, splits, relu):
    """Shapes for which the launcher gives each CTA two 128-row tiles of A sharing every B
    stage (M a multiple of 256 with at least 148 such blocks, or K of 64 steps or more):
    unsplit and split along K (17 slices of a 68-step K become 17 of 4 steps), with bias
    and ReLU."""
    lib, torch = env
    A, B, bias = _operands(torch, M, N, K, M + N + K + splits)
    out = torch.full((M, N), float("nan"), device="cuda")
    dA, dB, db = A.cuda(), B.cuda(), bias.cuda()
    if splits == 1:
        rc = lib.pdlp_tc_gemm(M, N, K, dA.data_ptr(), dB.data_ptr(), out.data_ptr(), db.data_ptr(), relu, None)
    else:
        ws = torch.empty(splits * M * N, device="cuda")
        rc = lib.pdlp_tc_gemm_split(M, N, K, dA.data_ptr(), dB.data_ptr(), out.data_ptr(), db.data_ptr(), relu,
                                    splits, ws.data_ptr(), None)
    assert rc == 0, lib.pdlp_last_error(None)
    ref, mag = _reference(A, B, bias, relu)
    tol = max(1e-5, K * 2.0 ** -24)
    assert np.all(np.abs(out.cpu().double().numpy() - ref) <= tol * mag + 1e-6)

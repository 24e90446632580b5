// Dense kernels of the learned warm start: the tcgen05 BF16 GEMM launcher and its
// C ABI test entry point.
#include <cuda_runtime.h>

#include <cstdio>
#include <string>

#include "pdlp.h"
#include "tc_gemm.cuh"

namespace pdlp {
void set_thread_error(const std::string& msg);

// Launches k_tc_gemm; returns a CUDA error code (cudaSuccess on success).
cudaError_t tc_gemm_launch(const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, __nv_bfloat16* Cb,
                           const float* bias, int M, int N, int K, int relu, int* err, cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemBytes);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  TcGemmArgs g{A, B, C, Cb, bias, M, N, K, relu, err};
  dim3 grid(N / kTcTile, M / kTcTile);
  k_tc_gemm<<<grid, 128, kTcSmemBytes, s>>>(g);
  return cudaGetLastError();
}
}  // namespace pdlp

extern "C" int pdlp_tc_gemm(int32_t M, int32_t N, int32_t K, const void* A, const void* B, float* C,
                            const float* bias, int32_t relu, void* stream) {
  using namespace pdlp;
  if (M <= 0 || N <= 0 || K <= 0 || M % kTcTile || N % kTcTile || K % kTcK) {
    set_thread_error("pdlp_tc_gemm: M, N must be positive multiples of 128 and K of 64");
    return PDLP_EINVAL;
  }
  if (!A || !B || !C) {
    set_thread_error("pdlp_tc_gemm: null array");
    return PDLP_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* err = nullptr;
  cudaError_t e = cudaMallocAsync(&err, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
  if (e == cudaSuccess)
    e = tc_gemm_launch(static_cast<const __nv_bfloat16*>(A), static_cast<const __nv_bfloat16*>(B), C, nullptr, bias,
                       M, N, K, relu, err, s);
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (err) cudaFreeAsync(err, s);
  if (e != cudaSuccess) {
    set_thread_error(std::string("pdlp_tc_gemm: ") + cudaGetErrorString(e));
    return PDLP_ECUDA;
  }
  if (herr) {
    set_thread_error("pdlp_tc_gemm: an mbarrier wait gave up (spin limit)");
    return PDLP_EINTERNAL;
  }
  return PDLP_OK;
}

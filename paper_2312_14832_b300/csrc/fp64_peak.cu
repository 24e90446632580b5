// fp64_peak: measures the FP64 fused multiply-add throughput of this GPU, the
// arithmetic roof of the FP64 PDHG kernels (every SpMV entry is one DFMA).
//
//   full  : every lane of every warp runs 8 independent DFMA chains
//   lane0 : the same kernel with one active lane per warp (the cost of a DFMA
//           instruction does not depend on the number of active lanes when the FP64
//           pipe is the limit, so its warp-instruction rate matches "full")
//
// Usage: fp64_peak [iters]   (default 32768 loop trips of 8 DFMAs per thread); prints one
// JSON line with lane-operations/s ("fma_per_s") and warp instructions/s.  Timing: CUDA
// events, best of 5 after one warm-up launch; grid = 8 CTAs of 256 threads per SM.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>

#define CK(x)                                                                        \
  do {                                                                               \
    cudaError_t e_ = (x);                                                            \
    if (e_ != cudaSuccess) {                                                         \
      fprintf(stderr, "CUDA error %s at line %d\n", cudaGetErrorString(e_), __LINE__); \
      return 1;                                                                      \
    }                                                                                \
  } while (0)

template <bool kOneLane>
__global__ void __launch_bounds__(256) k_dfma(double* out, long long iters, double a, double b) {
  if (kOneLane && (threadIdx.x & 31) != 0) return;
  double r[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) r[c] = 1e-3 * (threadIdx.x + c);
  for (long long i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) r[c] = fma(r[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += r[c];
  if (s == 123456.789) out[blockIdx.x] = s;   // keeps the chains live; never true here
}

int main(int argc, char** argv) {
  const long long iters = argc > 1 ? atoll(argv[1]) : 32768LL;
  if (iters < 1) {
    fprintf(stderr, "iters must be >= 1\n");
    return 2;
  }
  int sms = 0, dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8;
  double* out = nullptr;
  CK(cudaMalloc(&out, blocks * sizeof(double)));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best_full = 1e30f, best_one = 1e30f;
  const double a = 0.9999999, b = 1e-7;
  for (int rep = 0; rep < 6; ++rep) {
    float ms = 0.f;
    CK(cudaEventRecord(e0));
    k_dfma<false><<<blocks, 256>>>(out, iters, a, b);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0 && ms < best_full) best_full = ms;
    CK(cudaEventRecord(e0));
    k_dfma<true><<<blocks, 256>>>(out, iters, a, b);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0 && ms < best_one) best_one = ms;
  }
  CK(cudaGetLastError());
  const double warp_instr = (double)blocks * 8.0 * 8.0 * (double)iters;   // 8 warps per CTA, 8 chains
  const double full_s = best_full * 1e-3, one_s = best_one * 1e-3;
  printf("{\"sms\": %d, \"iters\": %lld, \"full_ms\": %.3f, \"fma_per_s\": %.4e, \"warp_instr_per_s\": %.4e, "
         "\"lane0_ms\": %.3f, \"lane0_warp_instr_per_s\": %.4e}\n",
         sms, iters, best_full, warp_instr * 32.0 / full_s, warp_instr / full_s, best_one, warp_instr / one_s);
  return 0;
}

// gather_ceiling: measures the two throughputs that bound the SpMV kernels on this GPU.
//
//   stream : coalesced read of values (8 B) and column indices (4 B) laid out like
//            the SELL-32 slots, no gather             -> GB/s
//   gather : the same stream plus x[col] for every entry from a vector of nx doubles
//            with uniformly random columns, FP64 FMA  -> gathers/s
//
// Usage: gather_ceiling [nnz] [nx]   (defaults 20000000 and 2000000); prints one JSON
// line.  Timing: CUDA events, best of 5 after one warm-up launch.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <vector>

#define CK(x)                                                                        \
  do {                                                                               \
    cudaError_t e_ = (x);                                                            \
    if (e_ != cudaSuccess) {                                                         \
      fprintf(stderr, "CUDA error %s at line %d\n", cudaGetErrorString(e_), __LINE__); \
      return 1;                                                                      \
    }                                                                                \
  } while (0)

constexpr int kSlotsPerWarp = 64;

__global__ void k_stream(const double* __restrict__ v, const int* __restrict__ c, long long nslots, double* out) {
  const int lane = threadIdx.x & 31;
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  long long s0 = w * kSlotsPerWarp, s1 = s0 + kSlotsPerWarp;
  if (s1 > nslots) s1 = nslots;
  unsigned long long a = 0;
  for (long long s = s0; s < s1; ++s)
    a ^= (unsigned long long)__double_as_longlong(__ldcs(v + s * 32 + lane)) + (unsigned)__ldcs(c + s * 32 + lane);
  if (s0 < s1) out[w * 32 + lane] = __longlong_as_double((long long)a);
}

__global__ void k_gather(const double* __restrict__ v, const int* __restrict__ c, const double* __restrict__ x,
                         long long nslots, double* out) {
  const int lane = threadIdx.x & 31;
  const long long w = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  long long s0 = w * kSlotsPerWarp, s1 = s0 + kSlotsPerWarp;
  if (s1 > nslots) s1 = nslots;
  double acc = 0.0;
  for (long long s = s0; s < s1; s += 4) {
    double vv[4], xv[4];
    int ci[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const long long e = (s + j < s1 ? s + j : s) * 32 + lane;
      vv[j] = __ldcs(v + e);
      ci[j] = __ldcs(c + e);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) xv[j] = __ldg(x + ci[j]);
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (s + j < s1) acc = fma(vv[j], xv[j], acc);
  }
  if (s0 < s1) out[w * 32 + lane] = acc;
}

int main(int argc, char** argv) {
  const long long nnz_req = argc > 1 ? atoll(argv[1]) : 20000000LL;
  const long long nx = argc > 2 ? atoll(argv[2]) : 2000000LL;
  if (nnz_req < 32 * kSlotsPerWarp || nx < 1) {
    fprintf(stderr, "need nnz >= %d and nx >= 1\n", 32 * kSlotsPerWarp);
    return 2;
  }
  const long long nslots = nnz_req / 32;
  const long long n = nslots * 32;
  const long long warps = (nslots + kSlotsPerWarp - 1) / kSlotsPerWarp;
  const int blocks = (int)((warps + 7) / 8);
  double *v = nullptr, *x = nullptr, *out = nullptr;
  int* c = nullptr;
  CK(cudaMalloc(&v, n * sizeof(double)));
  CK(cudaMalloc(&c, n * sizeof(int)));
  CK(cudaMalloc(&x, nx * sizeof(double)));
  CK(cudaMalloc(&out, warps * 32 * sizeof(double)));
  std::vector<int> hc((size_t)n);
  unsigned long long st = 0x9E3779B97F4A7C15ULL;
  for (long long i = 0; i < n; ++i) {  // splitmix-style stream of column indices
    st += 0x9E3779B97F4A7C15ULL;
    unsigned long long z = st;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    hc[(size_t)i] = (int)(z % (unsigned long long)nx);
  }
  CK(cudaMemcpy(c, hc.data(), n * sizeof(int), cudaMemcpyHostToDevice));
  CK(cudaMemset(v, 0, n * sizeof(double)));
  CK(cudaMemset(x, 0, nx * sizeof(double)));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best_s = 1e30f, best_g = 1e30f;
  for (int rep = 0; rep < 6; ++rep) {
    float ms = 0.f;
    CK(cudaEventRecord(e0));
    k_stream<<<blocks, 256>>>(v, c, nslots, out);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0 && ms < best_s) best_s = ms;
    CK(cudaEventRecord(e0));
    k_gather<<<blocks, 256>>>(v, c, x, nslots, out);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0 && ms < best_g) best_g = ms;
  }
  CK(cudaGetLastError());
  printf("{\"nnz\": %lld, \"nx\": %lld, \"stream_us\": %.2f, \"stream_gbs\": %.1f, \"gather_us\": %.2f, "
         "\"gathers_per_s\": %.4e, \"gather_algorithmic_gbs\": %.1f}\n",
         n, nx, best_s * 1e3, n * 12.0 / (best_s * 1e-3) / 1e9, best_g * 1e3, n / (best_g * 1e-3),
         (n * 12.0 + nx * 8.0) / (best_g * 1e-3) / 1e9);
  return 0;
}

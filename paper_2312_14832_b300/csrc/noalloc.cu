// pdlp_spmv_csr_noalloc: y = K x on the caller's device CSR arrays without any
// device allocation (declaration and contract in include/pdlp.h).
//
// Each thread takes a fixed run of kNoallocPerThread consecutive nonzeros and
// accumulates them with FMA (read through shared memory, see k_noalloc_runs).  A row that ends inside the run and also started
// inside it is written straight to y.  A row that crosses a run boundary leaves
// partial sums: the run where it starts (or any run it passes through) keeps a
// "tail" partial, the run where it ends keeps a "head" partial.  A second kernel
// adds, for each such row, the tails of the runs it crossed and its head, in run
// order, and writes zeros for empty rows.  The partials live in g_noalloc_scratch,
// a fixed device array of this file, so the call itself allocates nothing.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>

#include "pdlp.h"

namespace pdlp {
void set_thread_error(const std::string& msg);   // pdlp.cu: text for pdlp_last_error(NULL)
}

namespace {

constexpr int64_t kNoallocScratchBytes = 8ll << 20;   // 8 MiB held on every device that uses it
constexpr int64_t kNoallocPerThread = 64;             // nonzeros per thread
constexpr int64_t kBytesPerRun = 2 * sizeof(int32_t) + 2 * sizeof(double);
constexpr int64_t kMaxRuns = kNoallocScratchBytes / kBytesPerRun;
constexpr int kMaxDevices = 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

struct RunCarry {   // views into the scratch for `runs` runs
  int32_t* head_row;
  int32_t* tail_row;
  double* head_val;
  double* tail_val;
};

__host__ __device__ inline RunCarry carry_view(unsigned char* base, int64_t runs) {
  RunCarry c;
  c.head_val = reinterpret_cast<double*>(base);
  c.tail_val = c.head_val + runs;
  c.head_row = reinterpret_cast<int32_t*>(c.tail_val + runs);
  c.tail_row = c.head_row + runs;
  return c;
}

// Row holding nonzero position a (0 <= a < nnz): the last row r with row_ptr[r] <= a.
__device__ inline int64_t row_of(const int64_t* row_ptr, int64_t m, int64_t a) {
  int64_t lo = 0, hi = m;   // invariant: row_ptr[lo] <= a, answer in [lo, hi)
  while (hi - lo > 1) {
    int64_t mid = (lo + hi) >> 1;
    if (row_ptr[mid] <= a) lo = mid;
    else hi = mid;
  }
  return lo;
}

// One block of kRunsPerBlock threads takes kRunsPerBlock consecutive runs (a contiguous
// range of nonzeros).  The range is read in kPhases phases of kPhaseLen nonzeros per run:
// first the whole block loads the phase's values and column indices (each run's piece is
// kPhaseLen consecutive entries, so a warp's loads cover whole 32-byte sectors) and
// gathers x at those columns, every load independent of the others, into shared memory;
// then each thread walks its own piece in order, with the FMAs and row bookkeeping of a
// sequential run.  The arithmetic per run (one FMA per nonzero in index order) is the
// same as walking the run straight from global memory.
constexpr int kRunsPerBlock = 256;
constexpr int kPhaseLen = 8;
constexpr int kPhases = (int)(kNoallocPerThread / kPhaseLen);
constexpr int kPieceStride = kPhaseLen + 1;   // shared-memory stride of a run's piece (no bank conflicts)

__global__ void __launch_bounds__(kRunsPerBlock) k_noalloc_runs(int64_t m, int64_t nnz,
                                                                const int64_t* __restrict__ row_ptr,
                                                                const int32_t* __restrict__ col,
                                                                const double* __restrict__ val,
                                                                const double* __restrict__ x,
                                                                double* __restrict__ y, unsigned char* scratch,
                                                                int64_t runs) {
  __shared__ double sv[kRunsPerBlock * kPieceStride];
  __shared__ double sx[kRunsPerBlock * kPieceStride];
  const int64_t run0 = (int64_t)blockIdx.x * kRunsPerBlock;
  const int64_t t = run0 + threadIdx.x;
  const bool active = t < runs;
  const int64_t a = t * kNoallocPerThread;
  const int64_t b = active ? ((a + kNoallocPerThread < nnz) ? a + kNoallocPerThread : nnz) : a;
  int32_t head_row = -1, tail_row = -1;
  double head_val = 0.0, tail_val = 0.0;
  int64_t r = active ? row_of(row_ptr, m, a) : 0;
  int64_t rend = (active && r < m) ? row_ptr[r + 1] : 0;   // end of row r
  double acc = 0.0;
  for (int ph = 0; ph < kPhases; ++ph) {
    // stage: entry j of run (run0 + q) in this phase is nonzero run0*64 + 64 q + 8 ph + j
    int32_t c[kPhaseLen];
    double v[kPhaseLen];
#pragma unroll
    for (int i = 0; i < kPhaseLen; ++i) {
      const int idx = (int)threadIdx.x + i * kRunsPerBlock;
      const int q = idx / kPhaseLen, j = idx % kPhaseLen;
      const int64_t k = (run0 + q) * kNoallocPerThread + (int64_t)ph * kPhaseLen + j;
      c[i] = -1;
      v[i] = 0.0;
      if (k < nnz) {
        v[i] = __ldcs(val + k);
        c[i] = __ldcs(col + k);
      }
    }
#pragma unroll
    for (int i = 0; i < kPhaseLen; ++i) {
      const int idx = (int)threadIdx.x + i * kRunsPerBlock;
      const int q = idx / kPhaseLen, j = idx % kPhaseLen;
      sv[q * kPieceStride + j] = v[i];
      sx[q * kPieceStride + j] = c[i] >= 0 ? __ldg(x + c[i]) : 0.0;
    }
    __syncthreads();
    // walk: this thread's nonzeros a + 8 ph + j, j < 8, below b
    const int64_t k0 = a + (int64_t)ph * kPhaseLen;
#pragma unroll
    for (int j = 0; j < kPhaseLen; ++j) {
      const int64_t k = k0 + j;
      if (k < b) {
        acc = fma(sv[threadIdx.x * kPieceStride + j], sx[threadIdx.x * kPieceStride + j], acc);
        if (r < m && k + 1 == rend) {   // row r ends here
          if (row_ptr[r] >= a) {
            y[r] = acc;
          } else {
            head_row = (int32_t)r;
            head_val = acc;
          }
          acc = 0.0;
          ++r;
          while (r < m && row_ptr[r + 1] <= k + 1) ++r;   // skip empty rows
          rend = r < m ? row_ptr[r + 1] : 0;
        }
      }
    }
    __syncthreads();   // the next phase overwrites the staged entries
  }
  if (!active) return;
  RunCarry cv = carry_view(scratch, runs);
  if (r < m && b < row_ptr[r + 1] && row_ptr[r] < b) {   // row r continues past the run
    tail_row = (int32_t)r;
    tail_val = acc;
  }
  cv.head_row[t] = head_row;
  cv.head_val[t] = head_val;
  cv.tail_row[t] = tail_row;
  cv.tail_val[t] = tail_val;
}

__global__ void k_noalloc_fixup(int64_t m, const int64_t* __restrict__ row_ptr, double* __restrict__ y,
                                unsigned char* scratch, int64_t runs) {
  RunCarry cv = carry_view(scratch, runs);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < runs; t += stride) {
    const int32_t r = cv.head_row[t];
    if (r < 0) continue;
    int64_t j = t - 1;
    while (j >= 0 && cv.tail_row[j] == r) --j;   // runs j+1 .. t-1 carry tails of row r
    double s = 0.0;
    for (int64_t i = j + 1; i < t; ++i) s += cv.tail_val[i];
    y[r] = s + cv.head_val[t];
  }
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < m; r += stride)
    if (row_ptr[r] == row_ptr[r + 1]) y[r] = 0.0;
}

std::mutex g_noalloc_mutex;
unsigned char* g_noalloc_ptr[kMaxDevices] = {};

}  // namespace

extern "C" int pdlp_spmv_csr_noalloc(int64_t m, int64_t n, int64_t nnz, const int64_t* row_ptr,
                                     const int32_t* col_idx, const double* val, const double* x, double* y,
                                     void* stream) {
  if (m < 0 || n < 1 || nnz < 0 || m >= ((int64_t)1 << 31)) {
    pdlp::set_thread_error("pdlp_spmv_csr_noalloc: need m >= 0 (below 2^31), n >= 1, nnz >= 0");
    return PDLP_EINVAL;
  }
  const int64_t runs = (nnz + kNoallocPerThread - 1) / kNoallocPerThread;
  if (runs > kMaxRuns) {
    char buf[256];
    snprintf(buf, sizeof(buf),
             "pdlp_spmv_csr_noalloc: nnz = %lld exceeds the fixed scratch limit of %lld nonzeros",
             (long long)nnz, (long long)(kMaxRuns * kNoallocPerThread));
    pdlp::set_thread_error(buf);
    return PDLP_EINVAL;
  }
  if (m == 0) return PDLP_OK;
  if (!row_ptr || !y || (nnz > 0 && (!col_idx || !val || !x))) {
    pdlp::set_thread_error("pdlp_spmv_csr_noalloc: null array");
    return PDLP_EINVAL;
  }
  if (static_cast<const void*>(y) == static_cast<const void*>(x)) {
    pdlp::set_thread_error("pdlp_spmv_csr_noalloc: y must not overlap x (no in-place product)");
    return PDLP_EINVAL;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    pdlp::set_thread_error(std::string("pdlp_spmv_csr_noalloc: no current device: ") + cudaGetErrorString(e));
    return PDLP_ECUDA;
  }
  unsigned char* scratch = nullptr;
  {
    // once per device, with that device current: the device address of the array in the
    // device's primary context (the runtime's); it stays valid until the process exits
    // unless that context is destroyed (cudaDeviceReset)
    std::lock_guard<std::mutex> lk(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) {
        pdlp::set_thread_error(std::string("pdlp_spmv_csr_noalloc: cudaGetSymbolAddress failed: ") +
                               cudaGetErrorString(e));
        return PDLP_ECUDA;
      }
      g_noalloc_ptr[dev] = static_cast<unsigned char*>(p);
    }
    scratch = g_noalloc_ptr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (runs > 0) {
    const int64_t blocks = (runs + kRunsPerBlock - 1) / kRunsPerBlock;
    k_noalloc_runs<<<(unsigned)blocks, kRunsPerBlock, 0, s>>>(m, nnz, row_ptr, col_idx, val, x, y, scratch, runs);
  }
  int64_t fb = ((runs > m ? runs : m) + 255) / 256;
  if (fb > 148 * 8) fb = 148 * 8;
  if (fb < 1) fb = 1;
  k_noalloc_fixup<<<(unsigned)fb, 256, 0, s>>>(m, row_ptr, y, scratch, runs);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    pdlp::set_thread_error(std::string("pdlp_spmv_csr_noalloc: launch failed: ") + cudaGetErrorString(e));
    return PDLP_ECUDA;
  }
  return PDLP_OK;
}

// The learned warm start's network (an extension; the paper has no learned
// component): a 3-layer MLP  X -> relu(X W1' + b1) -> relu(. W2' + b2) -> . W3' + b3,
// BF16 operands on the tcgen05 tensor cores (tc_gemm.cuh) with FP32 accumulation,
// FP32 master weights, MSE loss and AdamW, forward and backward all on the device.
// Backward products use explicit BF16 transposes so that every GEMM is A * B'.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "pdlp.h"
#include "tc_gemm.cuh"

namespace pdlp {
void set_thread_error(const std::string& msg);

constexpr int kTcMaxDevices = 64;

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda).
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// Tensor map of a row-major BF16 matrix [rows x K] read in 128-row x 64-column boxes with
// 128-byte swizzle (the layout the MMA descriptors name).
static cudaError_t encode_operand(CUtensorMap* tm, const __nv_bfloat16* p, int rows, int K) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return cudaErrorNotSupported;
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)K * 2};
  cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)kTcTile};
  cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(p), dims, strides, box,
                         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Stages of the ring for products of few K steps per CTA (at most kTcShortK1 with one row
// tile, kTcShortK2 with two): a ring small enough for two CTAs per SM (97 KB), so that one
// CTA's epilogue overlaps another's loads.  Measured on the warm-start network's shapes:
// the output layer's weight gradient (60544 x 1024 x 256, one row tile) 0.217 -> 0.132 ms,
// its forward product (256 x 60544 x 1024, two row tiles) 0.097 -> 0.083 ms; the
// hidden-layer products (16 steps, one row tile) gain nothing from the smaller ring.
#ifndef PDLP_TC_SHORT_K1
#define PDLP_TC_SHORT_K1 4
#endif
#ifndef PDLP_TC_SHORT_K2
#define PDLP_TC_SHORT_K2 16
#endif
#ifndef PDLP_TC_SHORT_STAGES1
#define PDLP_TC_SHORT_STAGES1 3
#endif
#ifndef PDLP_TC_SHORT_STAGES2
#define PDLP_TC_SHORT_STAGES2 2
#endif
constexpr int kTcShortK1 = PDLP_TC_SHORT_K1;
constexpr int kTcShortK2 = PDLP_TC_SHORT_K2;
constexpr int kTcShortStages1 = PDLP_TC_SHORT_STAGES1;
constexpr int kTcShortStages2 = PDLP_TC_SHORT_STAGES2;

template <int kMT, int kSt>
static cudaError_t tc_gemm_attr() {
  return cudaFuncSetAttribute(k_tc_gemm<kMT, kSt>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              TcShape<kMT, kSt>::kSmem);
}

// The kernel's shared-memory opt-in, once per device (with that device current).
static cudaError_t tc_gemm_attrs() {
  static std::once_flag once[kTcMaxDevices];
  static cudaError_t res[kTcMaxDevices];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kTcMaxDevices) return cudaErrorInvalidDevice;
  std::call_once(once[dev], [&]() {
    res[dev] = tc_gemm_attr<1, 6>();
    if (res[dev] == cudaSuccess) res[dev] = tc_gemm_attr<2, 4>();
    if (res[dev] == cudaSuccess) res[dev] = tc_gemm_attr<1, kTcShortStages1>();
    if (res[dev] == cudaSuccess) res[dev] = tc_gemm_attr<2, kTcShortStages2>();
  });
  return res[dev];
}

// Row tiles per CTA: two 128-row tiles share each B stage when M allows it and the
// product has enough such blocks to fill the GPU, or a long K (where B, streamed once per
// block row, is most of the traffic and the split along K supplies the CTAs).
static int tc_gemm_mtiles(int M, int N, int K) {
  if (M % (2 * kTcTile)) return 1;
  const int blocks = (M / (2 * kTcTile)) * (N / kTcTile);
  return (blocks >= 148 || K / kTcK >= 64) ? 2 : 1;
}

// Slices of K for a product with few output tiles: enough CTAs for about two per SM,
// at least 8 steps of K per slice, at most max_splits.
int tc_gemm_splits(int M, int N, int K, int max_splits) {
  const int tiles = (M / (kTcTile * tc_gemm_mtiles(M, N, K))) * (N / kTcTile), kt = K / kTcK;
  if (tiles >= 148 || kt < 16 || max_splits <= 1) return 1;
  int sp = std::min(std::min(kt / 8, (2 * 148 + tiles - 1) / tiles), max_splits);
  sp = std::max(sp, 1);
  const int kps = (kt + sp - 1) / sp;
  return (kt + kps - 1) / kps;   // no empty slice
}

// C (FP32, optional) / Cb (BF16, optional) = A B' (+ bias, ReLU) with `splits` slices of K
// (1: no split; > 1: part holds splits x M x N floats).  Returns a CUDA error code.
cudaError_t tc_gemm_launch(const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, __nv_bfloat16* Cb,
                           const float* bias, int M, int N, int K, int relu, int splits, float* part, int* err,
                           cudaStream_t s, long long spin = kSpinLimit, int withhold = 0) {
  cudaError_t e = tc_gemm_attrs();
  if (e != cudaSuccess) return e;
  CUtensorMap ta, tb;
  e = encode_operand(&ta, A, M, K);
  if (e == cudaSuccess) e = encode_operand(&tb, B, N, K);
  if (e != cudaSuccess) return e;
  const int kt = K / kTcK;
  if (splits < 1 || !part) splits = 1;
  const int kps = (kt + splits - 1) / splits;
  splits = (kt + kps - 1) / kps;
  TcGemmArgs g{C, Cb, bias, splits > 1 ? part : nullptr, M, N, K, kps, relu, err, spin, withhold};
  const int mt = tc_gemm_mtiles(M, N, K);
  dim3 grid(N / kTcTile, M / (kTcTile * mt), splits);
  const bool short_k = kps <= (mt == 2 ? kTcShortK2 : kTcShortK1);
  if (mt == 2 && short_k)
    k_tc_gemm<2, kTcShortStages2><<<grid, 128, TcShape<2, kTcShortStages2>::kSmem, s>>>(ta, tb, g);
  else if (mt == 2)
    k_tc_gemm<2, 4><<<grid, 128, TcShape<2, 4>::kSmem, s>>>(ta, tb, g);
  else if (short_k)
    k_tc_gemm<1, kTcShortStages1><<<grid, 128, TcShape<1, kTcShortStages1>::kSmem, s>>>(ta, tb, g);
  else
    k_tc_gemm<1, 6><<<grid, 128, TcShape<1, 6>::kSmem, s>>>(ta, tb, g);
  e = cudaGetLastError();
  if (e == cudaSuccess && splits > 1) {
    const int64_t tot = (int64_t)M * N;
    const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 148 * 16);
    k_tc_splitk_reduce<<<blocks, 256, 0, s>>>(part, splits, M, N, bias, relu, C, Cb);
    e = cudaGetLastError();
  }
  return e;
}

// Error flag of the standalone entry points: one device int per GPU, its address looked
// up once per device.
__device__ int g_tc_gemm_err;
static int* tc_err_flag() {
  static std::mutex mu;
  static int* addr[kTcMaxDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kTcMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_tc_gemm_err) != cudaSuccess) return nullptr;
    addr[dev] = static_cast<int*>(p);
  }
  return addr[dev];
}

static int tc_gemm_entry(int32_t M, int32_t N, int32_t K, const void* A, const void* B, float* C, const float* bias,
                         int32_t relu, int32_t splits, float* workspace, void* stream, const char* name,
                         long long spin = kSpinLimit, int withhold = 0) {
  if (M <= 0 || N <= 0 || K <= 0 || M % kTcTile || N % kTcTile || K % kTcK) {
    set_thread_error(std::string(name) + ": M, N must be positive multiples of 128 and K of 64");
    return PDLP_EINVAL;
  }
  if (!A || !B || !C || (splits > 1 && !workspace) || splits < 1) {
    set_thread_error(std::string(name) + ": null array or bad split count");
    return PDLP_EINVAL;
  }
  if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15) {
    set_thread_error(std::string(name) + ": A and B must be 16-byte aligned");
    return PDLP_EINVAL;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int* err = tc_err_flag();
  if (!err) {
    set_thread_error(std::string(name) + ": no device error flag");
    return PDLP_ECUDA;
  }
  const int zero = 0;
  cudaError_t e = cudaMemcpyAsync(err, &zero, sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = tc_gemm_launch(static_cast<const __nv_bfloat16*>(A), static_cast<const __nv_bfloat16*>(B), C, nullptr, bias,
                       M, N, K, relu, splits, workspace, err, s, spin, withhold);
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_thread_error(std::string(name) + ": " + cudaGetErrorString(e));
    return PDLP_ECUDA;
  }
  if (herr) {
    set_thread_error(std::string(name) + ": an mbarrier wait gave up (spin limit)");
    return PDLP_ETIMEOUT;
  }
  return PDLP_OK;
}
}  // namespace pdlp

extern "C" int pdlp_tc_gemm(int32_t M, int32_t N, int32_t K, const void* A, const void* B, float* C,
                            const float* bias, int32_t relu, void* stream) {
  return pdlp::tc_gemm_entry(M, N, K, A, B, C, bias, relu, 1, nullptr, stream, "pdlp_tc_gemm");
}

extern "C" int pdlp_tc_gemm_wait_selftest(const void* A, const void* B, float* C, int64_t spin_limit, void* stream) {
  if (spin_limit < 1) {
    pdlp::set_thread_error("pdlp_tc_gemm_wait_selftest: spin_limit must be >= 1");
    return PDLP_EINVAL;
  }
  return pdlp::tc_gemm_entry(128, 128, 64, A, B, C, nullptr, 0, 1, nullptr, stream, "pdlp_tc_gemm_wait_selftest",
                             spin_limit, 1);
}

extern "C" int pdlp_tc_gemm_split(int32_t M, int32_t N, int32_t K, const void* A, const void* B, float* C,
                                  const float* bias, int32_t relu, int32_t splits, float* workspace, void* stream) {
  return pdlp::tc_gemm_entry(M, N, K, A, B, C, bias, relu, splits, workspace, stream, "pdlp_tc_gemm_split");
}

// ------------------------------------------------------------------ MLP kernels

namespace pdlp {

__global__ void k_mlp_fill_bf16_from_f32(__nv_bfloat16* dst, const float* src, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16_rn(src[i]);
}

// dst[R x Cp] (bf16) = src rows[idx[r]] (fp32, r < rows, c < cols), zero elsewhere.
__global__ void k_mlp_gather_rows(__nv_bfloat16* dst, int R, int Cp, const float* src, int cols, const int* idx,
                                  int rows) {
  const int64_t tot = (int64_t)R * Cp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(i / Cp), c = (int)(i % Cp);
    float v = 0.f;
    if (r < rows && c < cols) v = src[(int64_t)idx[r] * cols + c];
    dst[i] = __float2bfloat16_rn(v);
  }
}

// dst[C x R] = src[R x C]^T, 32x32 tiles through shared memory.
__global__ void k_mlp_transpose_bf16(__nv_bfloat16* dst, const __nv_bfloat16* src, int R, int C) {
  __shared__ __nv_bfloat16 t[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int r = by + j, c = bx + threadIdx.x;
    if (r < R && c < C) t[j][threadIdx.x] = src[(int64_t)r * C + c];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int c = bx + j, r = by + threadIdx.x;
    if (r < R && c < C) dst[(int64_t)c * R + r] = t[threadIdx.x][j];
  }
}

// dst[C x R] = src[R x C]^T for R a multiple of 16 and C of 64, without shared memory:
// warp w takes rows 16 (w / (C/64)) .. + 16 and columns 64 (w % (C/64)) .. + 64; lane l
// loads the column pair (2l, 2l + 1) of its 16 rows (4 bytes per row, 128 bytes per warp
// and row) and writes the two 32-byte output rows of that pair.
__global__ void k_mlp_transpose_bf16_w(__nv_bfloat16* dst, const __nv_bfloat16* src, int R, int C) {
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int cbs = C / 64;
  if (w >= (int64_t)(R / 16) * cbs) return;
  const int r0 = (int)(w / cbs) * 16, c0 = (int)(w % cbs) * 64 + 2 * lane;
  uint32_t v[16];
  const uint32_t* s32 = reinterpret_cast<const uint32_t*>(src);
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = s32[((int64_t)(r0 + k) * C + c0) >> 1];
  uint4 lo[2], hi[2];
  uint32_t* l32 = reinterpret_cast<uint32_t*>(lo);
  uint32_t* h32 = reinterpret_cast<uint32_t*>(hi);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    l32[j] = __byte_perm(v[2 * j], v[2 * j + 1], 0x5410);   // column c0: low halves of rows 2j, 2j+1
    h32[j] = __byte_perm(v[2 * j], v[2 * j + 1], 0x7632);   // column c0 + 1: high halves
  }
  uint4* d0 = reinterpret_cast<uint4*>(dst + (int64_t)c0 * R + r0);
  uint4* d1 = reinterpret_cast<uint4*>(dst + (int64_t)(c0 + 1) * R + r0);
  d0[0] = lo[0];
  d0[1] = lo[1];
  d1[0] = hi[0];
  d1[1] = hi[1];
}

// dY = (Y - T) / (rows * n_out) on the valid block, 0 elsewhere; BF16 copy; per-block
// partial sums of (Y - T)^2 for the loss.  Block (x, y) covers row y, columns x * 256 +
// threadIdx.x + k * 256 gridDim.x; a thread adds its squares in FP32, the block its
// threads' sums in FP64 in a fixed order; part[y * gridDim.x + x] = the block's sum.
__global__ void k_mlp_loss_grad(const float* Y, int Op, const float* T, int n_out, const int* idx, int rows,
                                float inv, float* dY, __nv_bfloat16* dYb, double* part) {
  const int r = blockIdx.y;
  const float* yr = Y + (size_t)r * Op;
  float* dyr = dY + (size_t)r * Op;
  __nv_bfloat16* dybr = dYb + (size_t)r * Op;
  const float* tr = r < rows ? T + (size_t)idx[r] * n_out : nullptr;
  float acc = 0.f;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < Op; c += gridDim.x * blockDim.x) {
    float g = 0.f;
    if (tr && c < n_out) {
      const float d = yr[c] - tr[c];
      acc = fmaf(d, d, acc);
      g = d * inv;
    }
    dyr[c] = g;
    dybr[c] = __float2bfloat16_rn(g);
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = (double)acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = sh[0];
}

// dZ = dH * (H > 0), FP32 and BF16.
__global__ void k_mlp_relu_back(float* dZ, __nv_bfloat16* dZb, const float* dH, const float* H, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float g = H[i] > 0.f ? dH[i] : 0.f;
    dZ[i] = g;
    dZb[i] = __float2bfloat16_rn(g);
  }
}

// db[c] = sum over rows r < R of dZ[r][c] (fixed row order).
__global__ void k_mlp_colsum(float* db, const float* dZ, int R, int C) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= C) return;
  float s = 0.f;
  for (int r = 0; r < R; ++r) s += dZ[(int64_t)r * C + c];
  db[c] = s;
}

// AdamW on one tensor: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// w -= lr (m_hat / (sqrt(v_hat) + eps) + wd w); wb (if not null) receives the BF16 copy
// of the new w that the next forward products read.
__global__ void k_mlp_adamw(float* w, float* m, float* v, const float* g, int64_t n, float lr, float wd, float b1,
                            float b2, float c1, float c2, float eps, __nv_bfloat16* wb) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wn = w[i] - lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * w[i]);
    w[i] = wn;
    if (wb) wb[i] = __float2bfloat16_rn(wn);
  }
}

// Loss of one minibatch from the per-block partial sums of k_mlp_loss_grad (one block of
// 256 threads: thread t adds part[t], part[t + 256], ... in order, then a fixed tree):
// out = sum(part[0..nb)) / denom, denom = 2 rows n_out.
__global__ void k_mlp_loss_total(const double* part, int nb, double denom, double* out) {
  __shared__ double sh[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += 256) s += part[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0] / denom;
}

}  // namespace pdlp

using namespace pdlp;

struct pdlp_mlp_ctx {
  int n_in, hid, n_out, in_p, out_p, maxb, bp;
  cudaStream_t s = nullptr;
  std::vector<void*> allocs;
  // parameters (FP32 masters), gradients, Adam moments: W1 [hid x in_p], W2 [hid x hid], W3 [out_p x hid]
  float *W[3], *b[3], *gW[3], *gb[3], *mW[3], *vW[3], *mb[3], *vb[3];
  int64_t wsz[3];
  int bsz[3];
  __nv_bfloat16 *Wb[3], *WTb[3];
  // activations for one batch
  __nv_bfloat16 *Xb, *XTb, *H1b, *H1Tb, *H2b, *H2Tb, *dYb, *dYTb, *dZ2b, *dZ2Tb, *dZ1Tb, *dZ1b;
  float *H1, *H2, *Y, *dY, *dH2, *dZ2, *dH1, *dZ1;
  double* part;
  int* err;
  float* gemm_ws = nullptr;   // partial products of GEMMs split along K
  int64_t gemm_ws_floats = 0;
  int* idx;          // batch row indices into the dataset
  float *dataX = nullptr, *dataT = nullptr;
  int64_t ndata = 0;
  int64_t step = 0;
  std::string msg;
};

namespace pdlp {

static int ceil_to(int v, int q) { return (v + q - 1) / q * q; }

template <class T>
static T* mlp_alloc(pdlp_mlp_ctx* h, size_t n) {
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T));
  if (e != cudaSuccess) throw std::string("cudaMalloc: ") + cudaGetErrorString(e);
  h->allocs.push_back(p);
  cudaMemsetAsync(p, 0, std::max<size_t>(n, 1) * sizeof(T), h->s);
  return (T*)p;
}

static void mlp_ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) throw std::string(what) + ": " + cudaGetErrorString(e);
}

static int gridn(int64_t n) { return (int)std::min<int64_t>(std::max<int64_t>((n + 255) / 256, 1), 148 * 8); }

constexpr int kMlpMaxSplits = 32;

static void gemm(pdlp_mlp_ctx* h, const __nv_bfloat16* A, const __nv_bfloat16* B, float* C, __nv_bfloat16* Cb,
                 const float* bias, int M, int N, int K, int relu) {
  int sp = tc_gemm_splits(M, N, K, kMlpMaxSplits);
  if ((int64_t)sp * M * N > h->gemm_ws_floats) sp = 1;
  mlp_ck(tc_gemm_launch(A, B, C, Cb, bias, M, N, K, relu, sp, h->gemm_ws, h->err, h->s), "tc_gemm");
}

static void transpose(pdlp_mlp_ctx* h, __nv_bfloat16* dst, const __nv_bfloat16* src, int R, int C) {
  if (R % 16 == 0 && C % 64 == 0 && ((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15) == 0) {
    const int64_t warps = (int64_t)(R / 16) * (C / 64);
    k_mlp_transpose_bf16_w<<<(unsigned)((warps + 7) / 8), 256, 0, h->s>>>(dst, src, R, C);
    return;
  }
  dim3 grid((C + 31) / 32, (R + 31) / 32), block(32, 8);
  k_mlp_transpose_bf16<<<grid, block, 0, h->s>>>(dst, src, R, C);
}

// Transposes of the BF16 W2, W3 for the backward products.
static void refresh_transposes(pdlp_mlp_ctx* h) {
  transpose(h, h->WTb[1], h->Wb[1], h->hid, h->hid);
  transpose(h, h->WTb[2], h->Wb[2], h->out_p, h->hid);
}

// BF16 copies of the weights and the transposes.
static void refresh_bf16(pdlp_mlp_ctx* h) {
  for (int l = 0; l < 3; ++l) k_mlp_fill_bf16_from_f32<<<gridn(h->wsz[l]), 256, 0, h->s>>>(h->Wb[l], h->W[l], h->wsz[l]);
  refresh_transposes(h);
}

// Forward on rows idx[0..rows) of X (device, n_in columns), outputs in h->Y.
static void forward(pdlp_mlp_ctx* h, const float* X, const int* idx, int rows) {
  k_mlp_gather_rows<<<gridn((int64_t)h->bp * h->in_p), 256, 0, h->s>>>(h->Xb, h->bp, h->in_p, X, h->n_in, idx, rows);
  gemm(h, h->Xb, h->Wb[0], h->H1, h->H1b, h->b[0], h->bp, h->hid, h->in_p, 1);
  gemm(h, h->H1b, h->Wb[1], h->H2, h->H2b, h->b[1], h->bp, h->hid, h->hid, 1);
  gemm(h, h->H2b, h->Wb[2], h->Y, nullptr, h->b[2], h->bp, h->out_p, h->hid, 0);
}

constexpr int kLossColBlocks = 8;   // column blocks of k_mlp_loss_grad per row

// Backward of the MSE loss against rows idx of T (device, n_out columns); gradients
// in h->gW / h->gb; the loss (sum of squares / (2 rows n_out)) goes to the device
// double *loss_dev.  Nothing is waited for.
static void backward_async(pdlp_mlp_ctx* h, const float* T, const int* idx, int rows, double* loss_dev) {
  const int nb = kLossColBlocks * h->bp;
  const float inv = (float)(1.0 / ((double)rows * h->n_out));
  k_mlp_loss_grad<<<dim3(kLossColBlocks, h->bp), 256, 0, h->s>>>(h->Y, h->out_p, T, h->n_out, idx, rows, inv, h->dY,
                                                                 h->dYb, h->part);
  transpose(h, h->dYTb, h->dYb, h->bp, h->out_p);
  transpose(h, h->H2Tb, h->H2b, h->bp, h->hid);
  transpose(h, h->H1Tb, h->H1b, h->bp, h->hid);
  transpose(h, h->XTb, h->Xb, h->bp, h->in_p);
  // layer 3
  gemm(h, h->dYTb, h->H2Tb, h->gW[2], nullptr, nullptr, h->out_p, h->hid, h->bp, 0);
  k_mlp_colsum<<<(h->out_p + 255) / 256, 256, 0, h->s>>>(h->gb[2], h->dY, h->bp, h->out_p);
  gemm(h, h->dYb, h->WTb[2], h->dH2, nullptr, nullptr, h->bp, h->hid, h->out_p, 0);
  k_mlp_relu_back<<<gridn((int64_t)h->bp * h->hid), 256, 0, h->s>>>(h->dZ2, h->dZ2b, h->dH2, h->H2,
                                                                    (int64_t)h->bp * h->hid);
  // layer 2
  transpose(h, h->dZ2Tb, h->dZ2b, h->bp, h->hid);
  gemm(h, h->dZ2Tb, h->H1Tb, h->gW[1], nullptr, nullptr, h->hid, h->hid, h->bp, 0);
  k_mlp_colsum<<<(h->hid + 255) / 256, 256, 0, h->s>>>(h->gb[1], h->dZ2, h->bp, h->hid);
  gemm(h, h->dZ2b, h->WTb[1], h->dH1, nullptr, nullptr, h->bp, h->hid, h->hid, 0);
  k_mlp_relu_back<<<gridn((int64_t)h->bp * h->hid), 256, 0, h->s>>>(h->dZ1, h->dZ1b, h->dH1, h->H1,
                                                                    (int64_t)h->bp * h->hid);
  // layer 1
  transpose(h, h->dZ1Tb, h->dZ1b, h->bp, h->hid);
  gemm(h, h->dZ1Tb, h->XTb, h->gW[0], nullptr, nullptr, h->hid, h->in_p, h->bp, 0);
  k_mlp_colsum<<<(h->hid + 255) / 256, 256, 0, h->s>>>(h->gb[0], h->dZ1, h->bp, h->hid);
  k_mlp_loss_total<<<1, 256, 0, h->s>>>(h->part, nb, 2.0 * rows * h->n_out, loss_dev);
  mlp_ck(cudaGetLastError(), "backward");
}

// backward_async, then the loss read back (one wait).
static double backward(pdlp_mlp_ctx* h, const float* T, const int* idx, int rows) {
  double* slot = h->part + (size_t)kLossColBlocks * h->bp;
  backward_async(h, T, idx, rows, slot);
  double L = 0.0;
  mlp_ck(cudaMemcpyAsync(&L, slot, sizeof(double), cudaMemcpyDeviceToHost, h->s), "loss copy");
  mlp_ck(cudaStreamSynchronize(h->s), "backward sync");
  return L;
}

static void check_err(pdlp_mlp_ctx* h) {
  int e = 0;
  mlp_ck(cudaMemcpyAsync(&e, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->s), "err copy");
  mlp_ck(cudaStreamSynchronize(h->s), "sync");
  if (e) throw std::string("tensor-core GEMM: an internal wait gave up");
}

template <class F>
static int mlp_guard(pdlp_mlp_ctx* h, F&& f) {
  if (!h) return PDLP_EINVAL;
  h->msg.clear();
  try {
    f();
    return PDLP_OK;
  } catch (const std::string& m) {
    h->msg = m;
    return m.rfind("bad", 0) == 0 ? PDLP_EINVAL : PDLP_ECUDA;
  } catch (...) {
    h->msg = "unexpected internal error";
    return PDLP_EINTERNAL;
  }
}

}  // namespace pdlp

extern "C" {

int pdlp_mlp_create(pdlp_mlp* out, int32_t n_in, int32_t hidden, int32_t n_out, int32_t max_batch) {
  if (!out) return PDLP_EINVAL;
  *out = nullptr;
  if (n_in < 1 || n_out < 1 || hidden < 128 || hidden % 128 || max_batch < 1) {
    set_thread_error("pdlp_mlp_create: need n_in, n_out >= 1, hidden a multiple of 128, max_batch >= 1");
    return PDLP_EINVAL;
  }
  pdlp_mlp_ctx* h = new pdlp_mlp_ctx();
  try {
    h->n_in = n_in;
    h->hid = hidden;
    h->n_out = n_out;
    h->in_p = ceil_to(n_in, 128);
    h->out_p = ceil_to(n_out, 128);
    h->maxb = max_batch;
    h->bp = ceil_to(max_batch, 128);
    mlp_ck(cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking), "stream");
    const int rows_of[3] = {h->hid, h->hid, h->out_p}, cols_of[3] = {h->in_p, h->hid, h->hid};
    for (int l = 0; l < 3; ++l) {
      h->wsz[l] = (int64_t)rows_of[l] * cols_of[l];
      h->bsz[l] = rows_of[l];
      for (float** p : {&h->W[l], &h->gW[l], &h->mW[l], &h->vW[l]}) *p = mlp_alloc<float>(h, h->wsz[l]);
      for (float** p : {&h->b[l], &h->gb[l], &h->mb[l], &h->vb[l]}) *p = mlp_alloc<float>(h, h->bsz[l]);
      h->Wb[l] = mlp_alloc<__nv_bfloat16>(h, h->wsz[l]);
      h->WTb[l] = mlp_alloc<__nv_bfloat16>(h, h->wsz[l]);
    }
    const int64_t bh = (int64_t)h->bp * h->hid;
    h->Xb = mlp_alloc<__nv_bfloat16>(h, (int64_t)h->bp * h->in_p);
    h->XTb = mlp_alloc<__nv_bfloat16>(h, (int64_t)h->bp * h->in_p);
    for (__nv_bfloat16** p : {&h->H1b, &h->H1Tb, &h->H2b, &h->H2Tb, &h->dZ2b, &h->dZ2Tb, &h->dZ1Tb, &h->dZ1b})
      *p = mlp_alloc<__nv_bfloat16>(h, bh);
    h->dYb = mlp_alloc<__nv_bfloat16>(h, (int64_t)h->bp * h->out_p);
    h->dYTb = mlp_alloc<__nv_bfloat16>(h, (int64_t)h->bp * h->out_p);
    for (float** p : {&h->H1, &h->H2, &h->dH2, &h->dZ2, &h->dH1, &h->dZ1}) *p = mlp_alloc<float>(h, bh);
    h->Y = mlp_alloc<float>(h, (int64_t)h->bp * h->out_p);
    h->dY = mlp_alloc<float>(h, (int64_t)h->bp * h->out_p);
    h->part = mlp_alloc<double>(h, (size_t)kLossColBlocks * h->bp + 1);   // per-block loss sums, then the loss
    h->err = mlp_alloc<int>(h, 1);
    // the split-K workspace of the largest split product of a training step
    const int shapes[8][3] = {{h->bp, h->hid, h->in_p},  {h->bp, h->hid, h->hid},  {h->bp, h->out_p, h->hid},
                              {h->out_p, h->hid, h->bp}, {h->bp, h->hid, h->out_p}, {h->hid, h->hid, h->bp},
                              {h->bp, h->hid, h->hid},   {h->hid, h->in_p, h->bp}};
    for (const auto& sh : shapes) {
      const int sp = tc_gemm_splits(sh[0], sh[1], sh[2], kMlpMaxSplits);
      if (sp > 1) h->gemm_ws_floats = std::max<int64_t>(h->gemm_ws_floats, (int64_t)sp * sh[0] * sh[1]);
    }
    if (h->gemm_ws_floats > 0) h->gemm_ws = mlp_alloc<float>(h, (size_t)h->gemm_ws_floats);
    h->idx = mlp_alloc<int>(h, h->bp);
    mlp_ck(cudaStreamSynchronize(h->s), "create");
  } catch (const std::string& m) {
    set_thread_error("pdlp_mlp_create: " + m);
    pdlp_mlp_free(h);
    return PDLP_ECUDA;
  }
  *out = h;
  return PDLP_OK;
}

void pdlp_mlp_free(pdlp_mlp h) {
  if (!h) return;
  if (h->s) cudaStreamSynchronize(h->s);
  for (void* p : h->allocs) cudaFree(p);
  if (h->s) cudaStreamDestroy(h->s);
  delete h;
}

const char* pdlp_mlp_last_error(pdlp_mlp h) { return h ? h->msg.c_str() : ""; }

int pdlp_mlp_set_params(pdlp_mlp h, const float* W1, const float* b1, const float* W2, const float* b2,
                        const float* W3, const float* b3) {
  return mlp_guard(h, [&]() {
    const float* Ws[3] = {W1, W2, W3};
    const float* bs[3] = {b1, b2, b3};
    const int rows[3] = {h->hid, h->hid, h->n_out}, cols[3] = {h->n_in, h->hid, h->hid};
    const int ldp[3] = {h->in_p, h->hid, h->hid};
    for (int l = 0; l < 3; ++l) {
      if (!Ws[l] || !bs[l]) throw std::string("bad: null parameter array");
      std::vector<float> w((size_t)h->wsz[l], 0.f), bb((size_t)h->bsz[l], 0.f);
      for (int r = 0; r < rows[l]; ++r)
        for (int c = 0; c < cols[l]; ++c) w[(size_t)r * ldp[l] + c] = Ws[l][(size_t)r * cols[l] + c];
      for (int r = 0; r < rows[l]; ++r) bb[(size_t)r] = bs[l][r];
      mlp_ck(cudaMemcpyAsync(h->W[l], w.data(), w.size() * 4, cudaMemcpyHostToDevice, h->s), "set W");
      mlp_ck(cudaMemcpyAsync(h->b[l], bb.data(), bb.size() * 4, cudaMemcpyHostToDevice, h->s), "set b");
      mlp_ck(cudaMemsetAsync(h->mW[l], 0, h->wsz[l] * 4, h->s), "zero m");
      mlp_ck(cudaMemsetAsync(h->vW[l], 0, h->wsz[l] * 4, h->s), "zero v");
      mlp_ck(cudaMemsetAsync(h->mb[l], 0, h->bsz[l] * 4, h->s), "zero m");
      mlp_ck(cudaMemsetAsync(h->vb[l], 0, h->bsz[l] * 4, h->s), "zero v");
      mlp_ck(cudaStreamSynchronize(h->s), "set params");
    }
    h->step = 0;
    refresh_bf16(h);
    mlp_ck(cudaStreamSynchronize(h->s), "set params");
  });
}

int pdlp_mlp_get_params(pdlp_mlp h, float* W1, float* b1, float* W2, float* b2, float* W3, float* b3) {
  return mlp_guard(h, [&]() {
    float* Ws[3] = {W1, W2, W3};
    float* bs[3] = {b1, b2, b3};
    const int rows[3] = {h->hid, h->hid, h->n_out}, cols[3] = {h->n_in, h->hid, h->hid};
    const int ldp[3] = {h->in_p, h->hid, h->hid};
    for (int l = 0; l < 3; ++l) {
      std::vector<float> w((size_t)h->wsz[l]), bb((size_t)h->bsz[l]);
      mlp_ck(cudaMemcpyAsync(w.data(), h->W[l], w.size() * 4, cudaMemcpyDeviceToHost, h->s), "get W");
      mlp_ck(cudaMemcpyAsync(bb.data(), h->b[l], bb.size() * 4, cudaMemcpyDeviceToHost, h->s), "get b");
      mlp_ck(cudaStreamSynchronize(h->s), "get params");
      if (Ws[l])
        for (int r = 0; r < rows[l]; ++r)
          for (int c = 0; c < cols[l]; ++c) Ws[l][(size_t)r * cols[l] + c] = w[(size_t)r * ldp[l] + c];
      if (bs[l])
        for (int r = 0; r < rows[l]; ++r) bs[l][r] = bb[(size_t)r];
    }
  });
}

int pdlp_mlp_load_data(pdlp_mlp h, int64_t count, const float* X, const float* T) {
  return mlp_guard(h, [&]() {
    if (count < 1 || !X) throw std::string("bad: empty data");
    if (h->dataX) {
      for (void* p : {(void*)h->dataX, (void*)h->dataT}) {
        auto it = std::find(h->allocs.begin(), h->allocs.end(), p);
        if (it != h->allocs.end()) {
          cudaFree(p);
          h->allocs.erase(it);
        }
      }
    }
    h->dataX = mlp_alloc<float>(h, (size_t)count * h->n_in);
    h->dataT = mlp_alloc<float>(h, (size_t)count * h->n_out);
    mlp_ck(cudaMemcpyAsync(h->dataX, X, (size_t)count * h->n_in * 4, cudaMemcpyHostToDevice, h->s), "data X");
    if (T) mlp_ck(cudaMemcpyAsync(h->dataT, T, (size_t)count * h->n_out * 4, cudaMemcpyHostToDevice, h->s), "data T");
    mlp_ck(cudaStreamSynchronize(h->s), "load data");
    h->ndata = count;
  });
}

int pdlp_mlp_forward(pdlp_mlp h, int32_t rows, const int32_t* idx, float* Y) {
  return mlp_guard(h, [&]() {
    if (!h->dataX || rows < 1 || rows > h->maxb || !idx || !Y) throw std::string("bad: forward arguments");
    for (int r = 0; r < rows; ++r)
      if (idx[r] < 0 || idx[r] >= h->ndata) throw std::string("bad: row index out of range");
    mlp_ck(cudaMemcpyAsync(h->idx, idx, sizeof(int) * rows, cudaMemcpyHostToDevice, h->s), "idx");
    forward(h, h->dataX, h->idx, rows);
    check_err(h);
    std::vector<float> y((size_t)h->bp * h->out_p);
    mlp_ck(cudaMemcpyAsync(y.data(), h->Y, y.size() * 4, cudaMemcpyDeviceToHost, h->s), "Y");
    mlp_ck(cudaStreamSynchronize(h->s), "forward");
    for (int r = 0; r < rows; ++r) std::memcpy(Y + (size_t)r * h->n_out, y.data() + (size_t)r * h->out_p, 4 * h->n_out);
  });
}

int pdlp_mlp_gradients(pdlp_mlp h, int32_t rows, const int32_t* idx, double* loss, float* gW1, float* gb1,
                       float* gW2, float* gb2, float* gW3, float* gb3) {
  return mlp_guard(h, [&]() {
    if (!h->dataX || rows < 1 || rows > h->maxb || !idx) throw std::string("bad: gradient arguments");
    for (int r = 0; r < rows; ++r)
      if (idx[r] < 0 || idx[r] >= h->ndata) throw std::string("bad: row index out of range");
    mlp_ck(cudaMemcpyAsync(h->idx, idx, sizeof(int) * rows, cudaMemcpyHostToDevice, h->s), "idx");
    forward(h, h->dataX, h->idx, rows);
    const double L = backward(h, h->dataT, h->idx, rows);
    check_err(h);
    if (loss) *loss = L;
    float* Ws[3] = {gW1, gW2, gW3};
    float* bs[3] = {gb1, gb2, gb3};
    const int nrows[3] = {h->hid, h->hid, h->n_out}, cols[3] = {h->n_in, h->hid, h->hid};
    const int ldp[3] = {h->in_p, h->hid, h->hid};
    for (int l = 0; l < 3; ++l) {
      std::vector<float> w((size_t)h->wsz[l]), bb((size_t)h->bsz[l]);
      mlp_ck(cudaMemcpyAsync(w.data(), h->gW[l], w.size() * 4, cudaMemcpyDeviceToHost, h->s), "gW");
      mlp_ck(cudaMemcpyAsync(bb.data(), h->gb[l], bb.size() * 4, cudaMemcpyDeviceToHost, h->s), "gb");
      mlp_ck(cudaStreamSynchronize(h->s), "gradients");
      if (Ws[l])
        for (int r = 0; r < nrows[l]; ++r)
          for (int c = 0; c < cols[l]; ++c) Ws[l][(size_t)r * cols[l] + c] = w[(size_t)r * ldp[l] + c];
      if (bs[l])
        for (int r = 0; r < nrows[l]; ++r) bs[l][r] = bb[(size_t)r];
    }
  });
}

int pdlp_mlp_train(pdlp_mlp h, int32_t epochs, int32_t batch, float lr, float weight_decay, uint64_t seed,
                   double* epoch_loss, double* train_ms) {
  return mlp_guard(h, [&]() {
    if (!h->dataX || epochs < 1 || batch < 1 || batch > h->maxb) throw std::string("bad: train arguments");
    const int64_t N = h->ndata;
    std::vector<int> perm((size_t)N);
    uint64_t st = seed * 0x9E3779B97F4A7C15ULL + 1;
    auto rnd = [&]() {
      st ^= st << 13;
      st ^= st >> 7;
      st ^= st << 17;
      return st;
    };
    cudaEvent_t e0, e1;
    mlp_ck(cudaEventCreate(&e0), "event");
    mlp_ck(cudaEventCreate(&e1), "event");
    float total_ms = 0.f;
    // the epoch's order and the minibatch losses stay on the device, so the steps of an
    // epoch are queued without waiting for one another
    const int64_t steps = N / batch;
    int* perm_dev = nullptr;
    double* loss_dev = nullptr;
    cudaError_t ae = cudaMalloc(&perm_dev, sizeof(int) * (size_t)std::max<int64_t>(N, 1));
    if (ae == cudaSuccess) ae = cudaMalloc(&loss_dev, sizeof(double) * (size_t)std::max<int64_t>(steps, 1));
    if (ae != cudaSuccess) {
      cudaFree(perm_dev);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      throw std::string("cudaMalloc: ") + cudaGetErrorString(ae);
    }
    std::vector<double> losses((size_t)std::max<int64_t>(steps, 1));
    try {
      for (int ep = 0; ep < epochs; ++ep) {
        for (int64_t i = 0; i < N; ++i) perm[(size_t)i] = (int)i;
        for (int64_t i = N - 1; i > 0; --i) std::swap(perm[(size_t)i], perm[(size_t)(rnd() % (uint64_t)(i + 1))]);
        mlp_ck(cudaMemcpyAsync(perm_dev, perm.data(), sizeof(int) * (size_t)N, cudaMemcpyHostToDevice, h->s), "perm");
        mlp_ck(cudaEventRecord(e0, h->s), "event");
        for (int64_t st_i = 0; st_i < steps; ++st_i) {
          const int* idx = perm_dev + st_i * batch;
          forward(h, h->dataX, idx, batch);
          backward_async(h, h->dataT, idx, batch, loss_dev + st_i);
          h->step += 1;
          const float b1 = 0.9f, b2 = 0.999f;
          const float c1 = 1.f - powf(b1, (float)h->step), c2 = 1.f - powf(b2, (float)h->step);
          for (int l = 0; l < 3; ++l) {
            k_mlp_adamw<<<gridn(h->wsz[l]), 256, 0, h->s>>>(h->W[l], h->mW[l], h->vW[l], h->gW[l], h->wsz[l], lr,
                                                             weight_decay, b1, b2, c1, c2, 1e-8f, h->Wb[l]);
            k_mlp_adamw<<<gridn(h->bsz[l]), 256, 0, h->s>>>(h->b[l], h->mb[l], h->vb[l], h->gb[l], h->bsz[l], lr,
                                                             0.f, b1, b2, c1, c2, 1e-8f, nullptr);
          }
          refresh_transposes(h);
        }
        mlp_ck(cudaGetLastError(), "train step");
        mlp_ck(cudaEventRecord(e1, h->s), "event");
        mlp_ck(cudaEventSynchronize(e1), "event");
        float ms = 0.f;
        mlp_ck(cudaEventElapsedTime(&ms, e0, e1), "event");
        total_ms += ms;
        double lsum = 0.0;
        if (steps > 0) {
          mlp_ck(cudaMemcpy(losses.data(), loss_dev, sizeof(double) * (size_t)steps, cudaMemcpyDeviceToHost),
                 "losses");
          for (int64_t i = 0; i < steps; ++i) lsum += losses[(size_t)i];
        }
        if (epoch_loss) epoch_loss[ep] = steps ? lsum / steps : 0.0;
      }
    } catch (...) {
      cudaFree(perm_dev);
      cudaFree(loss_dev);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      throw;
    }
    cudaFree(perm_dev);
    cudaFree(loss_dev);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    check_err(h);
    if (train_ms) *train_ms = total_ms;
  });
}

}  // extern "C"

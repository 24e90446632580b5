// BF16 GEMM on the 5th-generation tensor cores (tcgen05): C[M x N] = A[M x K] * B[N x K]^T
// with FP32 accumulation in tensor memory.  Used by the warm-start MLP (a dense
// contraction, unlike the LP's SpMV).
//
// One CTA of 128 threads computes a (128 kMT) x 128 block of C (kMT = 1 or 2 tiles of 128
// rows) over a range of K (all of K, or one slice of it when the product is split along
// K).  The roles are split:
//   - thread 0 is the producer: for each 64-wide step of K it waits until the MMAs have
//     released a stage of the ring, then has the tensor memory accelerator copy the kMT
//     128 x 64 tiles of A and the 128 x 64 tile of B into it (two-dimensional tiled
//     copies with 128-byte swizzle, the K-major layout the MMA descriptors name),
//     completing on the stage's "full" mbarrier;
//   - thread 32 issues the MMAs: it waits for a stage to be full, issues four
//     128x128x16 tcgen05.mma into each of the kMT TMEM accumulators (all reading the
//     stage's B tile), and tcgen05.commit's the stage's "empty" mbarrier, which hands the
//     stage back to the producer once those MMAs have read it; after the last step it
//     commits a "done" barrier;
//   - all four warps then run the epilogue: tcgen05.ld of each accumulator (warp w owns
//     TMEM lanes = rows 32w..32w+31), staged through shared memory so that every store
//     writes 128 consecutive bytes of a row of C, with bias and ReLU (or, for a slice of a
//     split product, the raw FP32 partial sums, which k_tc_splitk_reduce adds in slice
//     order).
// With kMT = 2 each B tile serves 256 rows of C, so B is streamed half as often; that is
// what bounds the warm-start network's wide products (B a 124 MB weight matrix, M = 256).
// The ring has kSt stages of 32 KB (kMT = 1) or 48 KB (kMT = 2): 6 or 4 (one CTA per SM,
// several copies in flight while the MMAs run), or, for few K steps per CTA, 3 or 2 (two
// CTAs per SM, one's epilogue overlapping the other's loads).  No multicast: every CTA
// copies its own tiles.
//
// Requirements (checked by the host launcher): M a multiple of 128 kMT, N a multiple of
// 128, K a multiple of 64, A and B row-major (K contiguous) with 16-byte aligned rows and
// bases.
// Every wait on an mbarrier gives up after kSpinLimit polls, sets *err and stops the
// CTA's pipeline; before the CTA leaves, the copies it issued are waited for (bounded)
// and its TMEM is freed.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cstdint>

namespace pdlp {

constexpr int kTcTile = 128;      // M and N of a CTA tile (and of one MMA)
constexpr int kTcK = 64;          // K per stage (128 bytes of BF16)
constexpr int kTcStageBytes = kTcTile * kTcK * 2;   // 16 KB per operand per stage
constexpr long long kSpinLimit = 1LL << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row groups
// 1024 bytes apart (SBO), version 1, start address in 16-byte units.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)(16 >> 4) << 16;     // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: D FP32, A and B BF16, both K-major, M = N = 128.
__device__ __forceinline__ uint32_t tc_idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcTile >> 3) << 17) | ((uint32_t)(kTcTile >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Waits for completion `parity` of the barrier; false after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, long long limit = kSpinLimit) {
  const uint32_t a = smem_u32(bar);
  for (long long i = 0; i < limit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

struct TcGemmArgs {
  float* C;                 // M x N (may be null)
  __nv_bfloat16* Cb;        // M x N BF16 copy (may be null)
  const float* bias;        // N (may be null)
  float* part;              // split product: gridDim.z x M x N partial sums (then C, Cb unused)
  int M, N, K;
  int ktiles;               // 64-wide steps of K per CTA (blockIdx.z takes steps z * ktiles ...)
  int relu;
  int* err;
  long long spin;           // poll limit of every mbarrier wait (kSpinLimit)
  int withhold;             // self-test of the bounded waits: issue no copy, so the first
                            // wait of the MMA thread can only give up
};

// Shape of one CTA of k_tc_gemm<kMT>: kMT 128-row tiles of A (kMT accumulators in
// TMEM, 128 columns each) share every 128 x 64 stage of B, so a CTA computes a
// (128 kMT) x 128 block of C and B is streamed once per 128 kMT rows of C.
template <int kMT, int kSt>
struct TcShape {
  static constexpr int kStages = kSt;
  static constexpr int kABytes = kMT * kTcStageBytes;       // A part of a stage
  static constexpr int kStageBytes = kABytes + kTcStageBytes;
  static constexpr int kSmem = kStages * kStageBytes + 1024;  // ring + alignment slack
  static constexpr int kTmemCols = kMT * kTcTile;
};

template <int kMT, int kSt>
__global__ void __launch_bounds__(128, 1) k_tc_gemm(const __grid_constant__ CUtensorMap tmA,
                                                    const __grid_constant__ CUtensorMap tmB, TcGemmArgs g) {
  using Sh = TcShape<kMT, kSt>;
  extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[kSt], empty[kSt], done;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int failed, issued_sh, consumed_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * (kMT * kTcTile), n0 = blockIdx.x * kTcTile;
  const int kt0 = blockIdx.z * g.ktiles;
  const int nk = min(g.ktiles, g.K / kTcK - kt0);
  // stage s: A rows m0 + 128 r at sA(s) + r * 16 KB (r < kMT), then B
  auto sA = [&](int s) { return base + (size_t)s * Sh::kStageBytes; };
  auto sB = [&](int s) { return base + (size_t)s * Sh::kStageBytes + Sh::kABytes; };

  if (threadIdx.x == 0) {
    for (int s = 0; s < kSt; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
    failed = 0;
    issued_sh = 0;
    consumed_sh = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                 "r"(Sh::kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;
  volatile int* vfailed = &failed;

  if (threadIdx.x == 0) {
    // producer: stage s = i % kSt; use i of a stage waits for the MMAs of use i - kSt
    int i = 0;
    for (; i < nk && !g.withhold; ++i) {
      const int s = i % kSt;
      if (i >= kSt && !mbar_wait(&empty[s], (uint32_t)(((i / kSt) - 1) & 1), g.spin)) {
        *vfailed = 1;
        break;
      }
      if (*vfailed) break;
      const uint32_t fb = smem_u32(&full[s]);
      const int kx = (kt0 + i) * kTcK;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(Sh::kStageBytes)
                   : "memory");
#pragma unroll
      for (int r = 0; r < kMT; ++r)
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
            "[%4];" ::"r"(smem_u32(sA(s) + r * kTcStageBytes)),
            "l"(reinterpret_cast<uint64_t>(&tmA)), "r"(kx), "r"(m0 + r * kTcTile), "r"(fb)
            : "memory");
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
          "[%4];" ::"r"(smem_u32(sB(s))),
          "l"(reinterpret_cast<uint64_t>(&tmB)), "r"(kx), "r"(n0), "r"(fb)
          : "memory");
    }
    issued_sh = i;
  } else if (threadIdx.x == 32) {
    // MMA issuer: per stage, four 16-deep steps of K into each of the kMT accumulators
    const uint32_t idesc = tc_idesc();
    int i = 0;
    for (; i < nk; ++i) {
      const int s = i % kSt;
      if (!mbar_wait(&full[s], (uint32_t)((i / kSt) & 1), g.spin)) {
        *vfailed = 1;
        break;
      }
      if (*vfailed) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(sA(s)), b0 = smem_u32(sB(s));
#pragma unroll
      for (int kk = 0; kk < kTcK / 16; ++kk) {
        const uint64_t bd = tc_desc(b0 + kk * 32);
        const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
#pragma unroll
        for (int r = 0; r < kMT; ++r) {
          const uint64_t ad = tc_desc(a0 + r * kTcStageBytes + kk * 32);
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + (uint32_t)(r * kTcTile)),
              "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
              : "memory");
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&empty[s]))
                   : "memory");
    }
    consumed_sh = i;
    // completes once every MMA issued above has finished
    if (i > 0)
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&done))
                   : "memory");
  }
  __syncthreads();
  const int consumed = consumed_sh, issued = issued_sh;
  bool ok = !*vfailed && consumed == nk && nk > 0;
  if (consumed > 0 && !mbar_wait(&done, 0, g.spin)) ok = false;
  if (!ok && threadIdx.x == 0) {
    atomicExch(g.err, 1);
    // no copy may land after the CTA has left: wait (bounded) for the unconsumed ones
    for (int i = consumed; i < issued; ++i) mbar_wait(&full[i % kSt], (uint32_t)((i / kSt) & 1), g.spin);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    // epilogue through shared memory (the ring is free: every copy has been consumed and
    // every MMA has finished): warp w stages a 32 x 32 block at a time; accumulator r
    // holds rows m0 + 128 r + (TMEM lane)
    float* tile = reinterpret_cast<float*>(base) + warp * 32 * 33;
    const size_t ldc = (size_t)g.N;
    for (int r = 0; r < kMT; ++r) {
      const int row0 = m0 + r * kTcTile + warp * 32;
      for (int cb = 0; cb < kTcTile; cb += 32) {
        uint32_t v[32];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(r * kTcTile + cb);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
              "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 32; ++j) tile[lane * 33 + j] = __uint_as_float(v[j]);
        __syncwarp();
        const int col = n0 + cb + lane;
        if (g.part) {
          float* P = g.part + (size_t)blockIdx.z * g.M * ldc;
          for (int rr = 0; rr < 32; ++rr) P[(size_t)(row0 + rr) * ldc + col] = tile[rr * 33 + lane];
        } else {
          const float bv = g.bias ? g.bias[col] : 0.0f;
          for (int rr = 0; rr < 32; ++rr) {
            float x = tile[rr * 33 + lane] + bv;
            if (g.relu) x = fmaxf(x, 0.0f);
            const size_t o = (size_t)(row0 + rr) * ldc + col;
            if (g.C) g.C[o] = x;
            if (g.Cb) g.Cb[o] = __float2bfloat16_rn(x);
          }
        }
        __syncwarp();
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Sh::kTmemCols) : "memory");
}

// C = sum over the splits of the partial products, in split order, + bias, ReLU.
__global__ void k_tc_splitk_reduce(const float* __restrict__ part, int splits, int M, int N,
                                   const float* __restrict__ bias, int relu, float* C, __nv_bfloat16* Cb) {
  const int64_t tot = (int64_t)M * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    float v = part[i];
    for (int z = 1; z < splits; ++z) v += part[(int64_t)z * tot + i];
    if (bias) v += bias[i % N];
    if (relu) v = fmaxf(v, 0.0f);
    if (C) C[i] = v;
    if (Cb) Cb[i] = __float2bfloat16_rn(v);
  }
}

}  // namespace pdlp

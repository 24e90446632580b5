// BF16 GEMM on the 5th-generation tensor cores (tcgen05): C[M x N] = A[M x K] * B[N x K]^T
// with FP32 accumulation in tensor memory.  Used by the warm-start MLP (a dense
// contraction, unlike the LP's SpMV).
//
// One CTA of 128 threads computes one 128 x 128 tile of C over a range of K (all of K,
// or one slice of it when the product is split along K).  The roles are split:
//   - thread 0 is the producer: for each 64-wide step of K it waits until the MMAs have
//     released a stage of the ring, then has the tensor memory accelerator copy the
//     128 x 64 tiles of A and B into it (two-dimensional tiled copies with 128-byte
//     swizzle, the K-major layout the MMA descriptors name), completing on the stage's
//     "full" mbarrier;
//   - thread 32 issues the MMAs: it waits for a stage to be full, issues four
//     128x128x16 tcgen05.mma into the TMEM accumulator, and tcgen05.commit's the stage's
//     "empty" mbarrier, which hands the stage back to the producer once those MMAs have
//     read it; after the last step it commits a "done" barrier;
//   - all four warps then run the epilogue: tcgen05.ld of the accumulator (warp w owns
//     TMEM lanes = rows 32w..32w+31), staged through shared memory so that every store
//     writes 128 consecutive bytes of a row of C, with bias and ReLU (or, for a slice of a
//     split product, the raw FP32 partial sums, which k_tc_splitk_reduce adds in slice
//     order).
// The ring has kTmStages stages of 32 KB (A and B), so up to kTmStages - 1 copies are in
// flight while the MMAs run.  No multicast: every CTA copies its own tiles.
//
// Requirements (checked by the host launcher): M, N multiples of 128, K a multiple of 64,
// A and B row-major (K contiguous) with 16-byte aligned rows and bases.
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
constexpr int kTmStages = 6;
constexpr int kTmSmemBytes = kTmStages * 2 * kTcStageBytes + 1024;   // ring + alignment slack
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

__global__ void __launch_bounds__(128, 1) k_tc_gemm(const __grid_constant__ CUtensorMap tmA,
                                                    const __grid_constant__ CUtensorMap tmB, TcGemmArgs g) {
  extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
  uint8_t* base = reinterpret_cast<uint8_t*>(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full[kTmStages], empty[kTmStages], done;
  __shared__ uint32_t tmem_base_sh;
  __shared__ int failed, issued_sh, consumed_sh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kTcTile, n0 = blockIdx.x * kTcTile;
  const int kt0 = blockIdx.z * g.ktiles;
  const int nk = min(g.ktiles, g.K / kTcK - kt0);
  auto sA = [&](int s) { return base + (size_t)s * 2 * kTcStageBytes; };
  auto sB = [&](int s) { return base + (size_t)s * 2 * kTcStageBytes + kTcStageBytes; };

  if (threadIdx.x == 0) {
    for (int s = 0; s < kTmStages; ++s) {
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
                 "r"(kTcTile)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base_sh;
  volatile int* vfailed = &failed;

  if (threadIdx.x == 0) {
    // producer: stage s = i % kTmStages; use i of a stage waits for the MMAs of use i - kTmStages
    int i = 0;
    for (; i < nk && !g.withhold; ++i) {
      const int s = i % kTmStages;
      if (i >= kTmStages && !mbar_wait(&empty[s], (uint32_t)(((i / kTmStages) - 1) & 1), g.spin)) {
        *vfailed = 1;
        break;
      }
      if (*vfailed) break;
      const uint32_t fb = smem_u32(&full[s]);
      const int kx = (kt0 + i) * kTcK;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(2 * kTcStageBytes)
                   : "memory");
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
          "[%4];" ::"r"(smem_u32(sA(s))),
          "l"(reinterpret_cast<uint64_t>(&tmA)), "r"(kx), "r"(m0), "r"(fb)
          : "memory");
      asm volatile(
          "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
          "[%4];" ::"r"(smem_u32(sB(s))),
          "l"(reinterpret_cast<uint64_t>(&tmB)), "r"(kx), "r"(n0), "r"(fb)
          : "memory");
    }
    issued_sh = i;
  } else if (threadIdx.x == 32) {
    // MMA issuer
    const uint32_t idesc = tc_idesc();
    int i = 0;
    for (; i < nk; ++i) {
      const int s = i % kTmStages;
      if (!mbar_wait(&full[s], (uint32_t)((i / kTmStages) & 1), g.spin)) {
        *vfailed = 1;
        break;
      }
      if (*vfailed) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(sA(s)), b0 = smem_u32(sB(s));
#pragma unroll
      for (int kk = 0; kk < kTcK / 16; ++kk) {
        const uint64_t ad = tc_desc(a0 + kk * 32), bd = tc_desc(b0 + kk * 32);
        const uint32_t acc = (i > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
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
    for (int i = consumed; i < issued; ++i)
      mbar_wait(&full[i % kTmStages], (uint32_t)((i / kTmStages) & 1), g.spin);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok) {
    // epilogue through shared memory (the ring is free: every copy has been consumed and
    // every MMA has finished): warp w stages a 32 x 32 block at a time
    float* tile = reinterpret_cast<float*>(base) + warp * 32 * 33;
    const size_t ldc = (size_t)g.N;
    for (int cb = 0; cb < kTcTile; cb += 32) {
      uint32_t r[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
            "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int j = 0; j < 32; ++j) tile[lane * 33 + j] = __uint_as_float(r[j]);
      __syncwarp();
      const int col = n0 + cb + lane;
      if (g.part) {
        float* P = g.part + (size_t)blockIdx.z * g.M * ldc;
        for (int rr = 0; rr < 32; ++rr) P[(size_t)(m0 + warp * 32 + rr) * ldc + col] = tile[rr * 33 + lane];
      } else {
        const float bv = g.bias ? g.bias[col] : 0.0f;
        for (int rr = 0; rr < 32; ++rr) {
          float v = tile[rr * 33 + lane] + bv;
          if (g.relu) v = fmaxf(v, 0.0f);
          const size_t o = (size_t)(m0 + warp * 32 + rr) * ldc + col;
          if (g.C) g.C[o] = v;
          if (g.Cb) g.Cb[o] = __float2bfloat16_rn(v);
        }
      }
      __syncwarp();
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTile) : "memory");
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

// BF16 GEMM on the 5th-generation tensor cores (tcgen05): C[M x N] = A[M x K] * B[N x K]^T
// with FP32 accumulation in tensor memory.  Used by the warm-start MLP (a dense
// contraction, unlike the LP's SpMV).
//
// One CTA of 128 threads computes one 128 x 128 tile of C.  K is walked in steps of
// 64 (one 128-byte row of BF16 per operand row); each step is staged in shared memory
// in the 128-byte-swizzled K-major layout the MMA reads, double buffered, and consumed
// by four 128x128x16 MMAs issued by one thread.  tcgen05.commit signals an mbarrier
// when a step's MMAs are done, which frees its buffer.  The epilogue reads the
// accumulator back with tcgen05.ld (each warp owns 32 rows = 32 TMEM lanes), adds an
// optional bias per column, applies an optional ReLU and writes FP32 and/or BF16.
//
// Requirements (checked by the host launcher): M, N multiples of 128, K a multiple of
// 64, A and B row-major (K contiguous) with 16-byte aligned rows.
// Every wait on an mbarrier gives up after kSpinLimit polls, sets *err and skips the
// remaining MMAs, so a fault in the pipeline ends the kernel instead of hanging it.
#pragma once
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

// Waits for completion `parity` of the barrier; false after kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long long i = 0; i < kSpinLimit; ++i) {
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

// 128 threads copy a 128-row x 64-column BF16 tile (row stride ld elements) into the
// swizzled layout: the 16-byte chunk c of row r lands at r*128 + ((c ^ (r & 7)) * 16).
__device__ __forceinline__ void tc_stage_tile(uint8_t* dst, const __nv_bfloat16* src, int ld) {
  for (int i = threadIdx.x; i < kTcTile * 8; i += blockDim.x) {
    const int r = i >> 3, c = i & 7;
    const uint4 v = *reinterpret_cast<const uint4*>(src + (size_t)r * ld + c * 8);
    *reinterpret_cast<uint4*>(dst + r * 128 + ((c ^ (r & 7)) << 4)) = v;
  }
}

struct TcGemmArgs {
  const __nv_bfloat16* A;   // M x K
  const __nv_bfloat16* B;   // N x K
  float* C;                 // M x N (may be null)
  __nv_bfloat16* Cb;        // M x N BF16 copy (may be null)
  const float* bias;        // N (may be null)
  int M, N, K;
  int relu;
  int* err;
};

__global__ void __launch_bounds__(128) k_tc_gemm(TcGemmArgs g) {
  extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
  // 1024-byte aligned stage buffers: [A0 B0 A1 B1]
  uint8_t* base = reinterpret_cast<uint8_t*>(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* sA[2] = {base, base + 2 * kTcStageBytes};
  uint8_t* sB[2] = {base + kTcStageBytes, base + 3 * kTcStageBytes};
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t tmem_base_sh;
  __shared__ int failed;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kTcTile, n0 = blockIdx.x * kTcTile;

  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    failed = 0;
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
  const uint32_t idesc = tc_idesc();
  const int nk = g.K / kTcK;

  for (int kt = 0; kt < nk; ++kt) {
    const int s = kt & 1;
    if (kt >= 2 && !failed) {
      // buffer s was last read by the MMAs of step kt-2 (completion number (kt-2)/2 of bar[s])
      if (!mbar_wait(&bar[s], (uint32_t)(((kt - 2) >> 1) & 1))) failed = 1;
    }
    __syncthreads();
    if (failed) break;
    tc_stage_tile(sA[s], g.A + (size_t)m0 * g.K + kt * kTcK, g.K);
    tc_stage_tile(sB[s], g.B + (size_t)n0 * g.K + kt * kTcK, g.K);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(sA[s]), b0 = smem_u32(sB[s]);
#pragma unroll
      for (int kk = 0; kk < kTcK / 16; ++kk) {
        const uint64_t ad = tc_desc(a0 + kk * 32), bd = tc_desc(b0 + kk * 32);
        const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&bar[s]))
                   : "memory");
    }
  }
  // the last commit covers every MMA issued before it
  if (!failed && nk > 0) {
    const int last = nk - 1;
    if (!mbar_wait(&bar[last & 1], (uint32_t)((last >> 1) & 1))) failed = 1;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!failed) {
    const int row = m0 + warp * 32 + lane;
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
      for (int j = 0; j < 32; ++j) {
        const int col = n0 + cb + j;
        float v = __uint_as_float(r[j]);
        if (g.bias) v += g.bias[col];
        if (g.relu) v = fmaxf(v, 0.0f);
        if (g.C) g.C[(size_t)row * g.N + col] = v;
        if (g.Cb) g.Cb[(size_t)row * g.N + col] = __float2bfloat16_rn(v);
      }
    }
  } else {
    // give the MMAs already issued a bounded chance to finish before TMEM is freed
    if (threadIdx.x == 0) {
      atomicExch(g.err, 1);
      if (nk > 0) {
        mbar_wait(&bar[0], 0);
        mbar_wait(&bar[1], 0);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTile) : "memory");
}

constexpr int kTcSmemBytes = 4 * kTcStageBytes + 1024;   // stages + alignment slack

}  // namespace pdlp

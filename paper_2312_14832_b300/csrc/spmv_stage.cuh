// SELL-32 row sums with the value / index stream staged in shared memory by the bulk-copy
// engine (one-dimensional cp.async.bulk from this GPU's global memory, no tensor map, no
// multicast), for the FP64 products of Section 2's primal and dual updates.
//
// sell_rows_kernel reads each slot's 32 values and 32 column indices with coalesced
// global loads, through the same load/store unit and L1 as the random gathers of the
// vector, which are what bounds the product (one distinct cache line per lane).  Here
// each warp instead copies its task's slots [s0, s1) into a ring of kNS buffers of kSB
// slots (values and indices), each buffer guarded by an mbarrier, kNS - 1 buffers ahead
// of the one it reads, so the load/store unit serves only the gathers and the
// epilogue's per-row operands.  The arithmetic is sell_rows_kernel's, in the same
// order: for a given task plan the two kernels give bit-identical results.
//
// Every mbarrier wait gives up after kStageSpin polls: the kernel then sets *err,
// stops waiting (the sums become garbage; the host reports PDLP_ETIMEOUT and retires
// the handle), and before the warp exits it waits, again with a limit, for every copy
// it issued, so that no copy lands in shared memory after the warp has left.
#pragma once
#include "kernels.cuh"

namespace pdlp {

constexpr long long kStageSpin = 1LL << 22;
constexpr int kStageBytesPerSlot = 32 * 8 + 32 * 4;   // values + column indices of one slot

// Shared memory of one warp's ring, and of a 256-thread CTA (8 warps).
template <int kSB, int kNS>
struct StageShape {
  static constexpr int kValBytes = kNS * kSB * 32 * 8;
  static constexpr int kColBytes = kNS * kSB * 32 * 4;
  static constexpr int kWarpBytes = kValBytes + kColBytes + 16 * ((kNS * 8 + 15) / 16);
  static constexpr int kCtaBytes = 8 * kWarpBytes;
};

__device__ __forceinline__ uint32_t stage_saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ bool stage_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool stage_wait(uint32_t bar, uint32_t parity) {
  for (long long i = 0; i < kStageSpin; ++i)
    if (stage_try_wait(bar, parity)) return true;
  return false;
}

// The ring of one warp over the slots [s0, s1) of its task.  Stage i holds slots
// [s0 + i kSB, s0 + (i + 1) kSB) in buffer i % kNS, completed on barrier i % kNS in phase
// (i / kNS) & 1.  All members are warp-uniform.
template <int kSB, int kNS>
struct StageRing {
  const double* gval;
  const int32_t* gcol;
  double* sval;
  int32_t* scol;
  uint32_t bar0;   // shared address of barrier 0 (barrier b at bar0 + 8 b)
  int s0, s1, nst;
  int cur;         // stage whose buffer is being read (-1 before the first)
  int issued;      // stages requested so far
  bool failed;
  int* err;

  __device__ __forceinline__ void issue(int i, int lane) {
    if (lane == 0) {
      const int a = s0 + i * kSB;
      const int ns = min(kSB, s1 - a);
      const int b = i % kNS;
      const uint32_t bar = bar0 + 8u * (uint32_t)b;
      const uint32_t vbytes = (uint32_t)ns * 256u, cbytes = (uint32_t)ns * 128u;
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(vbytes + cbytes)
                   : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              stage_saddr(sval + (size_t)b * kSB * 32)),
          "l"(gval + (size_t)a * 32), "r"(vbytes), "r"(bar)
          : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              stage_saddr(scol + (size_t)b * kSB * 32)),
          "l"(gcol + (size_t)a * 32), "r"(cbytes), "r"(bar)
          : "memory");
    }
    ++issued;
  }

  __device__ __forceinline__ void start(unsigned char* area, const double* v, const int32_t* c, int a, int e, int lane, int* errp) {
    using S = StageShape<kSB, kNS>;
    gval = v;
    gcol = c;
    sval = reinterpret_cast<double*>(area);
    scol = reinterpret_cast<int32_t*>(area + S::kValBytes);
    bar0 = stage_saddr(area + S::kValBytes + S::kColBytes);
    s0 = a;
    s1 = e;
    nst = (e - a + kSB - 1) / kSB;
    cur = -1;
    issued = 0;
    failed = false;
    err = errp;
    if (lane == 0) {
      for (int b = 0; b < kNS; ++b)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8u * (uint32_t)b) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    for (int i = 0; i < kNS && i < nst; ++i) issue(i, lane);
  }

  // Makes slot k (warp-uniform, read in increasing order) readable.
  __device__ __forceinline__ void ensure(int k, int lane) {
    const int i = (k - s0) / kSB;
    if (i == cur) return;
    if (cur >= 0 && cur + kNS < nst) {
      // every lane has read buffer cur % kNS: hand it to the copy of stage cur + kNS
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncwarp();
      if (!failed) issue(cur + kNS, lane);
    }
    cur = i;
    if (failed) return;
    if (!stage_wait(bar0 + 8u * (uint32_t)(i % kNS), (uint32_t)((i / kNS) & 1))) {
      failed = true;
      if (lane == 0) atomicExch(err, 1);
    }
  }

  __device__ __forceinline__ double val(int k, int lane) const {
    return sval[(size_t)((k - s0) % (kSB * kNS)) * 32 + lane];
  }
  __device__ __forceinline__ int32_t col(int k, int lane) const {
    return scol[(size_t)((k - s0) % (kSB * kNS)) * 32 + lane];
  }

  // Before the warp leaves: every copy it issued has landed (bounded waits).  In a
  // normal run every issued stage has been waited for and this does nothing.
  __device__ __forceinline__ void finish() {
    for (int i = cur + 1; i < issued; ++i) stage_wait(bar0 + 8u * (uint32_t)(i % kNS), (uint32_t)((i / kNS) & 1));
  }
};

// Sum of slots [s, e) of one chunk for this lane's row, values and indices from the ring;
// the same batching and order as chunk_sum.
template <class Op, int kBatch, int kSB, int kNS>
__device__ __forceinline__ double chunk_sum_staged(StageRing<kSB, kNS>& R, const double* __restrict__ xg, int s,
                                                   int e, int lane) {
  double acc = 0.0;
  for (int k = s; k < e; k += kBatch) {
    const int nb = min(kBatch, e - k);
    double v[kBatch], xv[kBatch];
    int ci[kBatch];
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
      if (j < nb) {
        R.ensure(k + j, lane);
        v[j] = R.val(k + j, lane);
        ci[j] = R.col(k + j, lane);
      }
    }
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
      xv[j] = 0.0;
      if (j < nb) xv[j] = __ldg(xg + ci[j]);
    }
#pragma unroll
    for (int j = 0; j < kBatch; ++j)
      if (j < nb) acc = Op::step(acc, v[j], xv[j]);
  }
  return acc;
}

// sell_rows_kernel with the staged stream (FP64 values, gathered products only).
// Dynamic shared memory: StageShape<kSB, kNS>::kCtaBytes; 256 threads.  With 8-slot
// buffers, two buffers per warp leave room for four CTAs per SM and three for three,
// and the register budget follows.
template <class Op, class Epi, int kBatch, int kSB, int kNS>
__global__ void __launch_bounds__(256, kNS <= 2 ? 4 : 3) sell_rows_staged_kernel(SellView A, const double* __restrict__ xg, Epi epi,
                                                               const DevState* __restrict__ st, int* err) {
  static_assert(Op::kGather, "the staged kernel computes gathered products");
  static_assert((kSB & (kSB - 1)) == 0, "kSB is a power of two");
  extern __shared__ __align__(128) unsigned char stage_smem[];
  if (st != nullptr && st->done) return;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int w = (int)(blockIdx.x * 8u) + wib;
  if (w >= A.ntasks) return;
  const SellTask Tk = A.tasks[w];
  epi.prepare(st);
  StageRing<kSB, kNS> R;
  R.start(stage_smem + (size_t)wib * StageShape<kSB, kNS>::kWarpBytes, A.val, A.col, Tk.s0, Tk.s1, lane, err);
  if (Tk.np == 0) {
    const int cb = A.chunk_ptr[min(Tk.chunk + lane, A.nchunks)];
    for (int j = 0; j < Tk.nc; ++j) {
      const int s = __shfl_sync(0xffffffffu, cb, j);
      const int e = __shfl_sync(0xffffffffu, cb, j + 1);
      const int row = (Tk.chunk + j) * 32 + lane;
      const typename Epi::Pre pre = epi.load(row);
      double acc = chunk_sum_staged<Op, kBatch>(R, xg, s, e, lane);
      if (Tk.wide) acc = wide_total<Op>(acc, lane);
      epi.finish(row, acc, pre);
    }
    R.finish();
    epi.task_end(w, lane);
  } else {
    const double acc = chunk_sum_staged<Op, kBatch>(R, xg, Tk.s0, Tk.s1, lane);
    R.finish();
    const int row = Tk.chunk * 32 + lane;
    A.gpart[(size_t)w * 32 + lane] = acc;
    __threadfence();
    int old = 0;
    if (lane == 0) old = atomicAdd(A.cnt + Tk.t0, 1);
    old = __shfl_sync(0xffffffffu, old, 0);
    if (old == Tk.np - 1) {
      __threadfence();
      const typename Epi::Pre pre = epi.load(row);
      double sum = __ldcg(A.gpart + (size_t)Tk.t0 * 32 + lane);
      for (int i = 1; i < Tk.np; ++i) sum = join_of<Op>(sum, __ldcg(A.gpart + (size_t)(Tk.t0 + i) * 32 + lane));
      if (lane == 0) A.cnt[Tk.t0] = 0;
      if (Tk.wide) sum = wide_total<Op>(sum, lane);
      epi.finish(row, sum, pre);
    }
    epi.task_end(w, lane);
  }
}

}  // namespace pdlp

// Persistent batched restarted PDHG: many independent LPs in one launch.
//
// The batch is stored as one block-diagonal LP: every LP owns a contiguous, 32-aligned
// range of internal rows and columns, and its chunks in the SELL-32 layouts of K and
// K' (layout.h).  Each CTA takes LPs from a work queue (largest first) and runs the
// whole method of Section 2 on one LP at a time: the step size by power iteration,
// the PDHG iterations, and the checks with the restart rule and the termination
// tests, all without leaving the CTA.  The two iterates live in shared memory, so
// the random gathers of both SpMVs are shared-memory loads; the matrix and the other
// per-row vectors stream from global memory.  Phases are separated by barriers: the
// primal phase reads y and writes x, the dual phase reads x and writes y.
//
// A team of CTAs can share one LP (k_batch_solve<true>, a thread-block cluster of up
// to 16 CTAs): CTA r owns a contiguous range of the LP's SELL chunks of K (rows) and
// of K' (columns), balanced by slot count, and every CTA keeps a full replica of x
// and y in its shared memory.  An owner writes each new x_j (y_i) into all replicas
// through distributed shared memory, and a cluster barrier ends each phase, so the
// gathers of both SpMVs stay local.  Team-wide sums add the CTAs' partial sums in
// rank order in every CTA, so all CTAs take the same restart decisions and leave the
// loop together; the cluster barrier is the hardware barrier, not a spin.
#pragma once
#include <cooperative_groups.h>
#include "kernels.cuh"

namespace pdlp {

struct LpDesc {
  int32_t m, n, m1, pad0;   // rows, columns, equality rows
  int32_t kc0, kc1;         // chunks of K (rows of this LP)
  int32_t tc0, tc1;         // chunks of K' (columns of this LP)
  int64_t r0, c0;           // first internal row / column (multiples of 32)
  int32_t mpad, npad;       // padded row / column counts
};

struct BatchArgs {
  const LpDesc* desc;
  const int32_t* order;      // LPs in the order the queue hands them out
  int32_t count;
  int32_t* next;             // queue position (left at zero after the launch)
  const int32_t* k_cptr;     // K: chunk_ptr, col, val (rows)
  const int32_t* k_col;
  const double* k_val;
  const int32_t* t_cptr;     // K': chunk_ptr, col, val (columns)
  const int32_t* t_col;
  const double* t_val;
  const double *c, *l, *u, *q, *invDr, *invDc;   // scaled problem, internal order
  double *sx, *sy, *xa, *ya, *kxp, *g, *kx_a, *g_a;
  double *xout, *yout;       // returned point per LP (scaled, internal order)
  const double *x0, *y0;     // warm start (scaled, internal order) or null
  const double* omega0;      // initial primal weight per LP (<= 0: the default) or null
  DevState* st;              // per LP
  DevParams P;
  int check_every;
  long long max_iter;
  int power_iters;
  double step_scale, eta_fixed, omega_fixed;
  int xs_off, ys_off, red_off;   // offsets (doubles) of x, y and the reduction area in shared memory
  int part_off;                  // team partial sums (kPartBuf doubles)
  long long slice_iters;         // > 0: an LP stops (resumably) at the first check after this many
                                 // iterations in this launch
  int resume;                    // 1: every LP of the queue continues from its suspended state
  // FP32 iterations (k_batch_solve32): FP32 values, problem vectors, interval sums and K x
  const float *k_val32, *t_val32, *c32, *l32, *u32, *q32;
  float *sx32, *sy32, *kxp32;
  double switch_tol;             // FP32 until the FP64-measured error is <= this (or stalls)
  // iterates in global memory (LPs too large for shared-memory replicas): one copy per LP,
  // shared by the team, gathered through L2
  double *xg, *yg;
  float *xg32, *yg32;
  // one LP run for a single-LP handle: its current point at the end, its restart
  // iterations and check records (null for batches)
  double *xcur, *ycur;
  long long* restarts;       // restart iterations: the handle's list (single LP) or, for a
  long long restart_stride;  // batch, restart_stride entries per LP (P.restart_cap of them kept)
  CheckRecord* log;
};

constexpr int kMaxTeam = 16;                         // CTAs per LP (non-portable cluster size)
constexpr int kPartStride = 16;                      // >= the widest team sum (10 values)
constexpr int kPartBuf = 2 * kMaxTeam * kPartStride; // two alternating areas

// The CTAs that solve one LP: one CTA (kCl = false) or the CTAs of a cluster.
template <bool kCl>
struct Team {
  int rank = 0, size = 1;
  __device__ __forceinline__ void init() {
    if constexpr (kCl) {
      cooperative_groups::cluster_group c = cooperative_groups::this_cluster();
      rank = (int)c.block_rank();
      size = (int)c.num_blocks();
    }
  }
  // barrier of the team (release/acquire at cluster scope for a cluster)
  __device__ __forceinline__ void sync() const {
    if constexpr (kCl) cooperative_groups::this_cluster().sync();
    else __syncthreads();
  }
  template <class T>
  __device__ __forceinline__ T* at(T* p, int r) const {
    if constexpr (kCl) return cooperative_groups::this_cluster().map_shared_rank(p, (unsigned)r);
    else return p;
  }
  // a[i] = v in the replica of every CTA of the team
  template <class V>
  __device__ __forceinline__ void put(V* a, int i, V v) const {
    if constexpr (kCl) {
      for (int k = 0; k < size; ++k) {
        int r = rank + k;
        if (r >= size) r -= size;
        *at(a + i, r) = v;
      }
    } else {
      a[i] = v;
    }
  }
};

// First chunk of piece r when chunks [c0, c1) are cut into `size` pieces of about
// equal slot counts (piece r is [split_point(r), split_point(r + 1))).
__device__ __forceinline__ int split_point(const int32_t* __restrict__ cptr, int c0, int c1, int r, int size) {
  if (r <= 0) return c0;
  if (r >= size) return c1;
  const long long s0 = cptr[c0], s1 = cptr[c1];
  const long long target = s0 + (s1 - s0) * r / size;
  int lo = c0, hi = c1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (cptr[mid] < target) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// Gather source of a batched SpMV: the shared-memory x or y, or a global vector.
// Where a product gathers its vector from: the shared-memory replicas of x or y, a global
// vector read through L2 only (ld.global.cg: a team's other CTAs write it), or a global
// vector read through L1 as well (one CTA per LP: only this CTA writes the vector, and
// __syncthreads makes its own writes visible to its later loads).
enum BatchSrc { kSrcSmemX, kSrcSmemY, kSrcGlobal, kSrcGlobalL1 };

// Rows in chunks [c0, c1) of a SELL matrix (in global memory, or a slice staged in
// shared memory: kMatS); warp w of the CTA takes chunks c0+w,
// c0+w+nw, ...  Each lane sums its row, gathering src[col - base], then calls
// epi(local_row, sum), local_row counted from chunk cbase (the LP's first chunk).
// Loads of kBB slots are issued together.
#ifndef PDLP_BATCH_LOADS
#define PDLP_BATCH_LOADS 4
#endif
// CTAs per SM the register allocation is sized for.  The one-CTA-per-LP FP64 kernel is
// latency-bound and gains from a third CTA even with the register spills that brings
// (2048 planted LPs: 5.73 s -> 4.90 s); the FP32 kernel loses (4.49 s -> 6.47 s) and the
// cluster kernels lose a few per cent, so they keep two.
#ifndef PDLP_BATCH_MIN_BLOCKS
#define PDLP_BATCH_MIN_BLOCKS 3
#endif
// With the iterates in global memory shared memory holds only the reduction scratch, and
// the latency-bound kernels gain from a fourth CTA per SM despite the spills: 200 x 300
// transportation LPs to 1e-4 (3000-iteration cap), 512 / 1000 LPs FP64 4.18 / 6.69 s ->
// 2.89 / 5.72 s, FP32 4.18 / 6.50 s -> 2.61 / 4.95 s (64 LPs on teams of 4: 0.67 -> 0.79 s).
#ifndef PDLP_BATCH_CL_GLOB_MIN_BLOCKS
#define PDLP_BATCH_CL_GLOB_MIN_BLOCKS 4
#endif
#ifndef PDLP_BATCH_GLOB_MIN_BLOCKS
#define PDLP_BATCH_GLOB_MIN_BLOCKS 4
#endif
#ifndef PDLP_BATCH32_MIN_BLOCKS
#define PDLP_BATCH32_MIN_BLOCKS 2
#endif
#ifndef PDLP_BATCH32_GLOB_MIN_BLOCKS
#define PDLP_BATCH32_GLOB_MIN_BLOCKS 4   // FP32 kernel with the iterates in global memory (see above)
#endif
constexpr int kBB = PDLP_BATCH_LOADS;
// The row loops ask the L2 for the slots of the warp's next chunk while they work on the
// current one (cp.async.bulk.prefetch: no registers or shared memory held in flight).
#ifndef PDLP_BATCH_L2PF
#define PDLP_BATCH_L2PF 1
#endif
// At most this many slots of a chunk are prefetched.  Measured on 1024 planted LPs (FP64
// 4.07 -> 3.37 s, FP32 2.92 -> 2.32 s): 64 slots, or two chunks ahead, or the first chunk
// of the next phase as well, are all slower; 1024 slots is no faster.
constexpr int kPfSlots = 256;

// Bulk L2 prefetch of [p, p + bytes): p 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void l2_prefetch(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <int SRC, bool kMatS, class F>
__device__ __forceinline__ void batch_rows(const int32_t* __restrict__ cptr, const int32_t* __restrict__ col,
                                           const double* __restrict__ val, int c0, int c1, int cbase,
                                           int64_t base, const double* gsrc, const BatchArgs& A, F epi) {
  extern __shared__ double bsm[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double* xs = bsm + A.xs_off;
  const double* ys = bsm + A.ys_off;
  for (int ch = c0 + wid; ch < c1; ch += nw) {
    const int s0 = cptr[ch], s1 = cptr[ch + 1];
    double acc = 0.0;
    for (int s = s0; s < s1; s += kBB) {
      const int nb = min(kBB, s1 - s);
      double v[kBB], xv[kBB];
      int ci[kBB];
#pragma unroll
      for (int j = 0; j < kBB; ++j)
        if (j < nb) {
          if constexpr (kMatS) {
            v[j] = val[(size_t)(s + j) * 32 + lane];
            ci[j] = col[(size_t)(s + j) * 32 + lane] - (int)base;
          } else {
            v[j] = __ldcs(val + (size_t)(s + j) * 32 + lane);
            ci[j] = __ldcs(col + (size_t)(s + j) * 32 + lane) - (int)base;
          }
        }
#pragma unroll
      for (int j = 0; j < kBB; ++j) {
        xv[j] = 0.0;
        if (j < nb) {
          if (SRC == kSrcSmemX) xv[j] = xs[ci[j]];
          else if (SRC == kSrcSmemY) xv[j] = ys[ci[j]];
          else if (SRC == kSrcGlobalL1) xv[j] = gsrc[ci[j]];
          else xv[j] = __ldcg(gsrc + ci[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < kBB; ++j)
        if (j < nb) acc = fma(v[j], xv[j], acc);
    }
    epi((ch - cbase) * 32 + lane, acc);
  }
}

// batch_rows with the epilogue split in two: pre(row) issues the loads of the row's
// epilogue operands before the row's products (their latency overlaps the slot loop),
// epi(row, sum, pre) finishes it; the next chunk's bounds are loaded ahead as well.
template <int SRC, class Pre, class F>
__device__ __forceinline__ void batch_rows_p(const int32_t* __restrict__ cptr, const int32_t* __restrict__ col,
                                             const double* __restrict__ val, int c0, int c1, int cbase,
                                             int64_t base, const double* gsrc, const BatchArgs& A, Pre pre, F epi) {
  extern __shared__ double bsm[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double* xs = bsm + A.xs_off;
  const double* ys = bsm + A.ys_off;
  int ch = c0 + wid;
  int s0 = 0, s1 = 0;
  if (ch < c1) {
    s0 = cptr[ch];
    s1 = cptr[ch + 1];
  }
  for (; ch < c1; ch += nw) {
    const int row = (ch - cbase) * 32 + lane;
    const auto pv = pre(row);
    int n0 = 0, n1 = 0;
    if (ch + nw < c1) {
      n0 = cptr[ch + nw];
      n1 = cptr[ch + nw + 1];
    }
    if (PDLP_BATCH_L2PF && lane == 0 && n1 > n0) {
      const uint32_t ns = (uint32_t)min(n1 - n0, kPfSlots);
      l2_prefetch(val + (size_t)n0 * 32, ns * 256u);
      l2_prefetch(col + (size_t)n0 * 32, ns * 128u);
    }
    double acc = 0.0;
    for (int s = s0; s < s1; s += kBB) {
      const int nb = min(kBB, s1 - s);
      double v[kBB], xv[kBB];
      int ci[kBB];
#pragma unroll
      for (int j = 0; j < kBB; ++j)
        if (j < nb) {
          v[j] = __ldcs(val + (size_t)(s + j) * 32 + lane);
          ci[j] = __ldcs(col + (size_t)(s + j) * 32 + lane) - (int)base;
        }
#pragma unroll
      for (int j = 0; j < kBB; ++j) {
        xv[j] = 0.0;
        if (j < nb) {
          if (SRC == kSrcSmemX) xv[j] = xs[ci[j]];
          else if (SRC == kSrcSmemY) xv[j] = ys[ci[j]];
          else if (SRC == kSrcGlobalL1) xv[j] = gsrc[ci[j]];
          else xv[j] = __ldcg(gsrc + ci[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < kBB; ++j)
        if (j < nb) acc = fma(v[j], xv[j], acc);
    }
    epi(row, acc, pv);
    s0 = n0;
    s1 = n1;
  }
}

// batch_rows_p for short chunks (a few slots each, such as K' of a transportation LP,
// two entries per column): a warp takes kG consecutive chunks at once, loads the slots
// of all of them two at a time, then gathers, then adds each row's products in slot
// order (the per-row order of batch_rows_p, so the sums are bit-identical), and
// finishes the kG rows' epilogues.  This keeps kG times more loads in flight per warp and
// drops the predicated-off lanes of an 8-slot batch on a 2-slot chunk.  The kernels with
// global iterates spill at their 64 registers, and more chunks per group means more
// spilling: on 300 / 1000 transportation LPs (200 x 300, one CTA per LP) two chunks take
// 0.904 / 2.12 ms per iteration against 0.925 / 2.31 ms with four; batches of 8 or 16
// slots in the long-row loop, or loading the next group's chunk bounds ahead, were
// slower (0.95-0.98 / 2.15-2.74 ms).
constexpr int kGrp = 2;
template <int SRC, class Pre, class F>
__device__ __forceinline__ void batch_rows_pg(const int32_t* __restrict__ cptr, const int32_t* __restrict__ col,
                                              const double* __restrict__ val, int c0, int c1, int cbase,
                                              int64_t base, const double* gsrc, const BatchArgs& A, Pre pre, F epi) {
  extern __shared__ double bsm[];
  constexpr int kB = 2;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const double* xs = bsm + A.xs_off;
  const double* ys = bsm + A.ys_off;
  using PV = decltype(pre(0));
  for (int ch0 = c0 + wid * kGrp; ch0 < c1; ch0 += nw * kGrp) {
    int s[kGrp], len[kGrp];
    PV pv[kGrp];
    double acc[kGrp];
    int lmax = 0;
#pragma unroll
    for (int g = 0; g < kGrp; ++g) {
      const int ch = ch0 + g;
      s[g] = 0;
      len[g] = 0;
      acc[g] = 0.0;
      if (ch < c1) {
        s[g] = cptr[ch];
        len[g] = cptr[ch + 1] - s[g];
        pv[g] = pre((ch - cbase) * 32 + lane);
        lmax = max(lmax, len[g]);
      }
    }
    if (PDLP_BATCH_L2PF && lane == 0) {
      const int n0 = ch0 + nw * kGrp;
      if (n0 < c1) {
        const int n1 = min(n0 + kGrp, c1);
        const int a = cptr[n0], b = cptr[n1];
        if (b > a) {
          const uint32_t ns = (uint32_t)min(b - a, kPfSlots);
          l2_prefetch(val + (size_t)a * 32, ns * 256u);
          l2_prefetch(col + (size_t)a * 32, ns * 128u);
        }
      }
    }
    for (int k = 0; k < lmax; k += kB) {
      double v[kGrp][kB], xv[kGrp][kB];
      int ci[kGrp][kB];
#pragma unroll
      for (int g = 0; g < kGrp; ++g)
#pragma unroll
        for (int j = 0; j < kB; ++j)
          if (k + j < len[g]) {
            v[g][j] = __ldcs(val + (size_t)(s[g] + k + j) * 32 + lane);
            ci[g][j] = __ldcs(col + (size_t)(s[g] + k + j) * 32 + lane) - (int)base;
          }
#pragma unroll
      for (int g = 0; g < kGrp; ++g)
#pragma unroll
        for (int j = 0; j < kB; ++j) {
          xv[g][j] = 0.0;
          if (k + j < len[g]) {
            if (SRC == kSrcSmemX) xv[g][j] = xs[ci[g][j]];
            else if (SRC == kSrcSmemY) xv[g][j] = ys[ci[g][j]];
            else if (SRC == kSrcGlobalL1) xv[g][j] = gsrc[ci[g][j]];
            else xv[g][j] = __ldcg(gsrc + ci[g][j]);
          }
        }
#pragma unroll
      for (int g = 0; g < kGrp; ++g)
#pragma unroll
        for (int j = 0; j < kB; ++j)
          if (k + j < len[g]) acc[g] = fma(v[g][j], xv[g][j], acc[g]);
    }
#pragma unroll
    for (int g = 0; g < kGrp; ++g)
      if (ch0 + g < c1) epi((ch0 + g - cbase) * 32 + lane, acc[g], pv[g]);
  }
}

// Rows of this CTA's resident slice of a SELL matrix (shared memory): chunk ch spans
// elements [cp[ch], cp[ch + 1]) of val / goff (32 per slot, lane = row), goff holds
// the byte offset of each entry's gathered element within src.  Same summation order
// per row as batch_rows; epi(row0 + 32 ch + lane, sum).
template <class F>
__device__ __forceinline__ void rows_s(const int* __restrict__ cp, const double* __restrict__ val,
                                       const int* __restrict__ goff, int nch, int row0,
                                       const double* __restrict__ src, F epi) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const char* sb = reinterpret_cast<const char*>(src);
  for (int ch = wid; ch < nch; ch += nw) {
    int e = cp[ch] + lane;
    const int e1 = cp[ch + 1];
    double acc = 0.0;
    for (; e + 96 < e1; e += 128) {
      const double v0 = val[e], v1 = val[e + 32], v2 = val[e + 64], v3 = val[e + 96];
      const int o0 = goff[e], o1 = goff[e + 32], o2 = goff[e + 64], o3 = goff[e + 96];
      const double x0 = *reinterpret_cast<const double*>(sb + o0);
      const double x1 = *reinterpret_cast<const double*>(sb + o1);
      const double x2 = *reinterpret_cast<const double*>(sb + o2);
      const double x3 = *reinterpret_cast<const double*>(sb + o3);
      acc = fma(v0, x0, acc);
      acc = fma(v1, x1, acc);
      acc = fma(v2, x2, acc);
      acc = fma(v3, x3, acc);
    }
    for (; e < e1; e += 32) acc = fma(val[e], *reinterpret_cast<const double*>(sb + goff[e]), acc);
    epi(row0 + ch * 32 + lane, acc);
  }
}

// Deterministic CTA sum of NV values per thread into red[0..NV) (shared memory):
// warp shuffles, then warp partials added in warp order by the first NV threads.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    const double s = warp_sum(v[i]);
    if (lane == 0) red[NV + wid * NV + i] = s;
  }
  __syncthreads();
  if ((int)threadIdx.x < NV) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[NV + w * NV + threadIdx.x];
    red[threadIdx.x] = s;
  }
  __syncthreads();
}

// Sum over the team of NV values per thread into red[0..NV) of every CTA: the CTA
// partials (block_sum) are written into each CTA's partial area, then added in rank
// order, so every CTA holds the same totals.  The two partial areas alternate
// (`flip`); the team barrier inside the next sum keeps an area from being reused
// before every CTA has read it.
template <int NV, bool kCl>
__device__ __forceinline__ void team_sum(double (&v)[NV], double* red, double* part, int& flip, const Team<kCl>& T) {
  block_sum<NV>(v, red);
  if constexpr (kCl) {
    double* pa = part + flip * (kMaxTeam * kPartStride);
    flip ^= 1;
    const int tid = threadIdx.x;
    if (tid < NV) {
      const double s = red[tid];
      for (int r = 0; r < T.size; ++r) *T.at(pa + T.rank * kPartStride + tid, r) = s;
    }
    T.sync();
    if (tid < NV) {
      double s = 0.0;
      for (int r = 0; r < T.size; ++r) s += pa[r * kPartStride + tid];
      red[tid] = s;
    }
    __syncthreads();
  }
}

// Euclidean norm over the team of v[j0..j1) (each CTA passes its own range).
template <bool kCl>
__device__ __forceinline__ double team_norm(const double* v, int j0, int j1, double* red, double* part, int& flip,
                                            const Team<kCl>& T) {
  double a[1] = {0.0};
  for (int j = j0 + (int)threadIdx.x; j < j1; j += blockDim.x) a[0] = fma(v[j], v[j], a[0]);
  team_sum<1>(a, red, part, flip, T);
  return sqrt(red[0]);
}

// The 18 check quantities of the LP (same definitions as k_kkt_partials), reduced
// over the team into tot[0..NQ); this CTA adds rows [ir0, ir1) and columns [jc0, jc1).
// avg_is_cur: the average equals the current point.
template <bool kCl>
__device__ __forceinline__ void batch_kkt(const BatchArgs& A, const LpDesc& D, bool avg_is_cur, double it,
                                          double* red, double* tot, int ir0, int ir1, int jc0, int jc1,
                                          double* part, int& flip, const Team<kCl>& T, const double* xs,
                                          const double* ys) {
  // xs, ys: the current point of the LP (indices local to the LP; this CTA reads its own
  // rows and columns only)
  {
    double acc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = 0.0;
    const int i1 = min(ir1, D.m);
    for (int i = ir0 + (int)threadIdx.x; i < i1; i += blockDim.x) {
      const int64_t gi = D.r0 + i;
      const double qi = A.q[gi], id = A.invDr[gi], yai = A.ya[gi];
      const bool ineq = i >= D.m1;
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const bool avg = (p == 1) && !avg_is_cur;
        const double kx = avg ? A.kx_a[gi] : A.kxp[gi];
        const double yi = avg ? A.sy[gi] * it : ys[i];
        double r = kx - qi;
        if (ineq) r = min0(r);
        const double ru = r * id;
        acc[4 * p + 0] = fma(r, r, acc[4 * p + 0]);
        acc[4 * p + 1] = fma(ru, ru, acc[4 * p + 1]);
        acc[4 * p + 2] = fma(qi, yi, acc[4 * p + 2]);
        const double dy = yi - yai;
        acc[4 * p + 3] = fma(dy, dy, acc[4 * p + 3]);
      }
    }
    team_sum<8>(acc, red, part, flip, T);
    if ((int)threadIdx.x < 8) tot[threadIdx.x] = red[threadIdx.x];
    __syncthreads();
  }
  {
    double acc[10];
#pragma unroll
    for (int i = 0; i < 10; ++i) acc[i] = 0.0;
    const int j1 = min(jc1, D.n);
    for (int j = jc0 + (int)threadIdx.x; j < j1; j += blockDim.x) {
      const int64_t gj = D.c0 + j;
      const double cj = A.c[gj], lj = A.l[gj], uj = A.u[gj], id = A.invDc[gj], xaj = A.xa[gj];
      const bool lf = !is_neg_inf(lj), uf = !is_pos_inf(uj);
#pragma unroll
      for (int p = 0; p < 2; ++p) {
        const bool avg = (p == 1) && !avg_is_cur;
        const double g = avg ? A.g_a[gj] : A.g[gj];
        const double xj = avg ? A.sx[gj] * it : xs[j];
        const double d = cj - g;
        const bool neg = __double2hiint(d) < 0;
        double lam, rd;
        if (lf && uf) { lam = d; rd = 0.0; }
        else if (lf) { lam = neg ? 0.0 : d; rd = neg ? d : 0.0; }
        else if (uf) { lam = neg ? d : 0.0; rd = neg ? 0.0 : d; }
        else { lam = 0.0; rd = d; }
        const double rdu = rd * id;
        const double bnd = is_zero(lam) ? 0.0 : (__double2hiint(lam) < 0 ? uj : lj);
        acc[5 * p + 0] = fma(rd, rd, acc[5 * p + 0]);
        acc[5 * p + 1] = fma(rdu, rdu, acc[5 * p + 1]);
        acc[5 * p + 2] = fma(bnd, lam, acc[5 * p + 2]);
        acc[5 * p + 3] = fma(cj, xj, acc[5 * p + 3]);
        const double dx = xj - xaj;
        acc[5 * p + 4] = fma(dx, dx, acc[5 * p + 4]);
      }
    }
    team_sum<10>(acc, red, part, flip, T);
    if ((int)threadIdx.x < 10) tot[8 + threadIdx.x] = red[threadIdx.x];
    __syncthreads();
  }
}

// Shared-memory footprint (bytes) of one CTA's resident slice: its chunks of K and K'
// (chunk pointers, columns, values) and the per-entry vectors of the rows and columns
// it owns.  The host sizes the launch with the same formula.
__host__ __device__ inline long long resident_bytes(long long kch, long long kslots, long long tch, long long tslots,
                                                    long long rows, long long cols) {
  const long long dbl = 32 * (kslots + tslots) + 4 * cols + 3 * rows;
  const long long ints = 32 * (kslots + tslots) + (kch + 1) + (tch + 1);
  return 8 * dbl + 4 * ints + 16;
}

// Runs restarted PDHG on LP b with the team T (one CTA, or the CTAs of a cluster).
// kRes: the CTA's slice of K and K' and the vectors of its rows and columns are copied
// into shared memory first, so an iteration touches only shared memory (and, in a
// cluster, the replicas of the other CTAs); the running sums and K x are written back
// to global memory at every check.
// kGlob: the iterates live in global memory (A.xg, A.yg), one copy per LP shared by the
// team (each CTA writes only its own rows and columns, gathers go through L2).
template <bool kCl, bool kRes, bool kGlob>
__device__ void batch_solve_one(const BatchArgs& A, int b, const Team<kCl>& T) {
  static_assert(!(kRes && kGlob), "resident slices gather from shared-memory replicas");
  extern __shared__ double bsm[];
  const LpDesc& D0 = A.desc[b];
  double* xs = kGlob ? A.xg + D0.c0 : bsm + A.xs_off;
  double* ys = kGlob ? A.yg + D0.r0 : bsm + A.ys_off;
  double* red = bsm + A.red_off;
  double* part = bsm + A.part_off;
  __shared__ DevState S;
  __shared__ double tot[NQ];
  __shared__ double scal[4];
  const LpDesc D = A.desc[b];
  const int n = D.n, m = D.m;
  const int tid = threadIdx.x, nt = blockDim.x;
  int flip = 0;
  // this CTA's chunks of K (rows [ir0, ir1)) and of K' (columns [jc0, jc1))
  const int kr0 = split_point(A.k_cptr, D.kc0, D.kc1, T.rank, T.size);
  const int kr1 = split_point(A.k_cptr, D.kc0, D.kc1, T.rank + 1, T.size);
  const int tr0 = split_point(A.t_cptr, D.tc0, D.tc1, T.rank, T.size);
  const int tr1 = split_point(A.t_cptr, D.tc0, D.tc1, T.rank + 1, T.size);
  const int ir0 = (kr0 - D.kc0) * 32, ir1 = (kr1 - D.kc0) * 32;
  const int jc0 = (tr0 - D.tc0) * 32, jc1 = (tr1 - D.tc0) * 32;
  const int mo1 = min(ir1, m), no1 = min(jc1, n);
  // the entries of the iterates this CTA writes when it sets them all: its whole replica,
  // or (global iterates) its own rows and columns; then a barrier over the team
  const int xw0 = kGlob ? jc0 : 0, xw1 = kGlob ? jc1 : D.npad;
  const int yw0 = kGlob ? ir0 : 0, yw1 = kGlob ? ir1 : D.mpad;
  auto fill_sync = [&]() {
    if constexpr (kGlob) T.sync();
    else __syncthreads();
  };
  auto put = [&](double* a, int i, double v) {
    if constexpr (kGlob) a[i] = v;
    else T.put(a, i, v);
  };

  // per-entry vectors as the iterations see them: v[i - ofs]
  const double* cv = A.c + D.c0;
  const double* lv = A.l + D.c0;
  const double* uv = A.u + D.c0;
  double* sxv = A.sx + D.c0;
  const double* qv = A.q + D.r0;
  double* syv = A.sy + D.r0;
  double* kxv = A.kxp + D.r0;
  int jofs = 0, iofs = 0;
  // resident slices (shared memory): chunk pointers in elements, values, gather offsets
  const int* kpS = nullptr;
  const double* kvS = nullptr;
  const int* kgS = nullptr;
  const int* tpS = nullptr;
  const double* tvS = nullptr;
  const int* tgS = nullptr;
  if constexpr (kRes) {
    const int ks0 = A.k_cptr[kr0], ks1 = A.k_cptr[kr1], ts0 = A.t_cptr[tr0], ts1 = A.t_cptr[tr1];
    const int kn = 32 * (ks1 - ks0), tn = 32 * (ts1 - ts0);
    const int nco = jc1 - jc0, nro = ir1 - ir0;
    double* p = bsm + A.part_off + kPartBuf;
    double* kv = p; p += kn;
    double* tv = p; p += tn;
    double* cS = p; p += nco;
    double* lS = p; p += nco;
    double* uS = p; p += nco;
    double* sxS = p; p += nco;
    double* qS = p; p += nro;
    double* syS = p; p += nro;
    double* kxS = p; p += nro;
    int32_t* ip = reinterpret_cast<int32_t*>(p);
    int32_t* kg = ip; ip += kn;
    int32_t* tg = ip; ip += tn;
    int32_t* kp = ip; ip += (kr1 - kr0) + 1;
    int32_t* tp = ip;
    for (int e = tid; e < kn; e += nt) {
      kv[e] = A.k_val[(size_t)ks0 * 32 + e];
      kg[e] = (int)(A.k_col[(size_t)ks0 * 32 + e] - D.c0) * 8;
    }
    for (int e = tid; e < tn; e += nt) {
      tv[e] = A.t_val[(size_t)ts0 * 32 + e];
      tg[e] = (int)(A.t_col[(size_t)ts0 * 32 + e] - D.r0) * 8;
    }
    for (int e = tid; e <= kr1 - kr0; e += nt) kp[e] = (A.k_cptr[kr0 + e] - ks0) * 32;
    for (int e = tid; e <= tr1 - tr0; e += nt) tp[e] = (A.t_cptr[tr0 + e] - ts0) * 32;
    for (int j = tid; j < nco; j += nt) {
      const int64_t gj = D.c0 + jc0 + j;
      cS[j] = A.c[gj];
      lS[j] = A.l[gj];
      uS[j] = A.u[gj];
    }
    for (int i = tid; i < nro; i += nt) qS[i] = A.q[D.r0 + ir0 + i];
    if (A.resume) {
      for (int j = tid; j < nco; j += nt) sxS[j] = A.sx[D.c0 + jc0 + j];
      for (int i = tid; i < nro; i += nt) {
        syS[i] = A.sy[D.r0 + ir0 + i];
        kxS[i] = A.kxp[D.r0 + ir0 + i];
      }
    }
    kpS = kp;
    kvS = kv;
    kgS = kg;
    tpS = tp;
    tvS = tv;
    tgS = tg;
    cv = cS;
    lv = lS;
    uv = uS;
    sxv = sxS;
    qv = qS;
    syv = syS;
    kxv = kxS;
    jofs = jc0;
    iofs = ir0;
    __syncthreads();
  }
  // K times a vector over this CTA's rows (gathering x: the replica or a global vector
  // of the LP's columns), and K' times a vector over its columns
  auto Kmul = [&](bool from_replica, const double* gsrc, auto&& epi) {
    if constexpr (kRes) {
      if (from_replica) rows_s(kpS, kvS, kgS, kr1 - kr0, ir0, xs, epi);
      else rows_s(kpS, kvS, kgS, kr1 - kr0, ir0, gsrc, epi);
    } else if constexpr (kGlob) {
      batch_rows<kSrcGlobal, false>(A.k_cptr, A.k_col, A.k_val, kr0, kr1, D.kc0, D.c0, from_replica ? xs : gsrc, A,
                                    epi);
    } else {
      if (from_replica) batch_rows<kSrcSmemX, false>(A.k_cptr, A.k_col, A.k_val, kr0, kr1, D.kc0, D.c0, nullptr, A, epi);
      else batch_rows<kSrcGlobal, false>(A.k_cptr, A.k_col, A.k_val, kr0, kr1, D.kc0, D.c0, gsrc, A, epi);
    }
  };
  auto Tmul = [&](bool from_replica, const double* gsrc, auto&& epi) {
    if constexpr (kRes) {
      if (from_replica) rows_s(tpS, tvS, tgS, tr1 - tr0, jc0, ys, epi);
      else rows_s(tpS, tvS, tgS, tr1 - tr0, jc0, gsrc, epi);
    } else if constexpr (kGlob) {
      batch_rows<kSrcGlobal, false>(A.t_cptr, A.t_col, A.t_val, tr0, tr1, D.tc0, D.r0, from_replica ? ys : gsrc, A,
                                    epi);
    } else {
      if (from_replica) batch_rows<kSrcSmemY, false>(A.t_cptr, A.t_col, A.t_val, tr0, tr1, D.tc0, D.r0, nullptr, A, epi);
      else batch_rows<kSrcGlobal, false>(A.t_cptr, A.t_col, A.t_val, tr0, tr1, D.tc0, D.r0, gsrc, A, epi);
    }
  };

  // ---- step size: power iteration on K'K from v0 = 1/sqrt(n) (a resumed LP keeps its own)
  double eta = A.eta_fixed;
  if (!(eta > 0.0) && !A.resume) {
    const double v0 = 1.0 / sqrt((double)n);
    for (int j = xw0 + tid; j < xw1; j += nt) xs[j] = j < n ? v0 : 0.0;
    fill_sync();
    for (int it = 0; it < A.power_iters; ++it) {
      Kmul(true, nullptr,
                                  [&](int i, double s) { put(ys, i, s); });
      T.sync();
      Tmul(true, nullptr,
                                  [&](int j, double s) { A.g[D.c0 + j] = s; });
      __syncthreads();
      const double nw = team_norm(A.g + D.c0, jc0, jc1, red, part, flip, T);
      if (nw != 0.0)
        for (int j = jc0 + tid; j < jc1; j += nt) put(xs, j, A.g[D.c0 + j] / nw);
      T.sync();
    }
    Kmul(true, nullptr,
                                [&](int i, double s) { put(ys, i, s); });
    T.sync();
    const double sn = m > 0 ? team_norm(ys, ir0, ir1, red, part, flip, T) : 0.0;
    eta = sn > 0.0 ? A.step_scale / sn : 1.0;
  }
  // ---- initial primal weight ||c||/||q|| and the unscaled norms for termination
  double omega = A.omega_fixed;
  {
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = jc0 + tid; j < no1; j += nt) {
      const double cj = A.c[D.c0 + j];
      const double cu = cj * A.invDc[D.c0 + j];
      a[0] = fma(cj, cj, a[0]);
      a[2] = fma(cu, cu, a[2]);
    }
    for (int i = ir0 + tid; i < mo1; i += nt) {
      const double qi = A.q[D.r0 + i];
      const double qu = qi * A.invDr[D.r0 + i];
      a[1] = fma(qi, qi, a[1]);
      a[3] = fma(qu, qu, a[3]);
    }
    team_sum<4>(a, red, part, flip, T);
    if (tid == 0) {
      const double cn = sqrt(red[0]), qn = sqrt(red[1]);
      scal[0] = (cn > 1e-10 && qn > 1e-10) ? cn / qn : 1.0;
      scal[1] = sqrt(red[2]);
      scal[2] = sqrt(red[3]);
    }
    __syncthreads();
    if (!(omega > 0.0)) omega = scal[0];
    if (A.omega0 != nullptr && A.omega0[b] > 0.0) omega = A.omega0[b];
  }
  DevParams P = A.P;
  P.cnorm = scal[1];
  P.qnorm = scal[2];

  if (A.resume) {
    // ---- continue a suspended LP: its state, its current point (kept in xout / yout),
    // and the running sums, anchor and K x that stayed in global memory
    for (int j = xw0 + tid; j < xw1; j += nt) xs[j] = A.xout[D.c0 + j];
    for (int i = yw0 + tid; i < yw1; i += nt) ys[i] = A.yout[D.r0 + i];
    if (tid == 0) {
      S = A.st[b];
      S.suspended = 0;
    }
    fill_sync();
  } else {
    // ---- initial point (the warm start or 0, projected onto X and Y) and anchor; every
    // CTA fills its own replicas, the owners the per-entry vectors
    for (int j = xw0 + tid; j < xw1; j += nt) {
      const int64_t gj = D.c0 + j;
      const double x0 = j < n ? clamp_box(A.x0 ? A.x0[gj] : 0.0, A.l[gj], A.u[gj]) : 0.0;
      xs[j] = x0;
      if (j >= jc0 && j < jc1) {
        A.xa[gj] = x0;
        A.sx[gj] = 0.0;
        sxv[j - jofs] = 0.0;
      }
    }
    for (int i = yw0 + tid; i < yw1; i += nt) {
      const int64_t gi = D.r0 + i;
      double y0 = (A.y0 && i < m) ? A.y0[gi] : 0.0;
      if (i >= D.m1) y0 = max0(y0);
      ys[i] = y0;
      if (i >= ir0 && i < ir1) {
        A.ya[gi] = y0;
        A.sy[gi] = 0.0;
        syv[i - iofs] = 0.0;
      }
    }
    fill_sync();
    Kmul(true, nullptr, [&](int i, double s) {
      A.kxp[D.r0 + i] = s;
      kxv[i - iofs] = s;
    });
    Tmul(true, nullptr,
                                [&](int j, double s) { A.g[D.c0 + j] = s; });
    __syncthreads();
    if (tid == 0) {
      memset(&S, 0, sizeof(S));
      S.eta = eta;
      S.omega = omega;
      S.tau = eta / omega;
      S.sigma = eta * omega;
    }
    __syncthreads();
    batch_kkt(A, D, true, 0.0, red, tot, ir0, ir1, jc0, jc1, part, flip, T, xs, ys);
    if (tid == 0) {
      const double gap = tot[Q_QY_C] + tot[Q_LT_C] - tot[Q_CX_C];
      S.kkt_anchor = kkt_w(tot[Q_PRS_C], tot[Q_DRS_C], gap, S.omega);
      S.kkt_prev = __longlong_as_double(0x7FF0000000000000LL);
    }
    __syncthreads();
  }

  // ---- iterations (Section 2: primal step, dual step with extrapolation) and checks
  // short chunks (at most 4 slots on average over this CTA's range) go through the
  // grouped row loop (global iterates only)
  const bool short_t = kGlob && (A.t_cptr[tr1] - A.t_cptr[tr0]) <= 4 * (tr1 - tr0);
  const bool short_k = kGlob && (A.k_cptr[kr1] - A.k_cptr[kr0]) <= 4 * (kr1 - kr0);
  // the iterations' gathers from global iterates: through L1 when this CTA is the LP's
  // only writer
  constexpr int kGSrc = kCl ? kSrcGlobal : kSrcGlobalL1;
  long long k = S.k, t = S.t;
  const long long k_start = k;
  int until_check = A.check_every;
  for (;;) {
    const bool at_limit = k >= A.max_iter;
    if (!at_limit) {
      const double tau = S.tau, sigma = S.sigma;
      // primal step (Section 2) on g = K'y of this CTA's columns
      struct PreP { double c, l, u, sx, x; };
      auto pre_p = [&](int j) {
        const int jl = j - jofs;
        return PreP{cv[jl], lv[jl], uv[jl], sxv[jl], xs[j]};
      };
      auto epi_p = [&](int j, double gsum, const PreP& p) {
        const double xn = clamp_box(fma(-tau, p.c - gsum, p.x), p.l, p.u);
        put(xs, j, xn);
        sxv[j - jofs] = p.sx + xn;
      };
      if constexpr (kRes)
        Tmul(true, nullptr, [&](int j, double gsum) { epi_p(j, gsum, pre_p(j)); });
      else if constexpr (kGlob)
        if (short_t)
          batch_rows_pg<kGSrc>(A.t_cptr, A.t_col, A.t_val, tr0, tr1, D.tc0, D.r0, ys, A, pre_p, epi_p);
        else
          batch_rows_p<kGSrc>(A.t_cptr, A.t_col, A.t_val, tr0, tr1, D.tc0, D.r0, ys, A, pre_p, epi_p);
      else
        batch_rows_p<kSrcSmemY>(A.t_cptr, A.t_col, A.t_val, tr0, tr1, D.tc0, D.r0, nullptr, A, pre_p, epi_p);
      T.sync();
      // dual step with extrapolation (Section 2) on v = K x of this CTA's rows
      struct PreD { double q, kx, y, sy; };
      auto pre_d = [&](int i) {
        const int il = i - iofs;
        return PreD{qv[il], kxv[il], ys[i], syv[il]};
      };
      auto epi_d = [&](int i, double v, const PreD& p) {
        const double e = p.q + p.kx;
        double yn = fma(sigma, fma(-2.0, v, e), p.y);
        if (i >= D.m1) yn = max0(yn);
        put(ys, i, yn);
        syv[i - iofs] = p.sy + yn;
        kxv[i - iofs] = v;
      };
      if constexpr (kRes)
        Kmul(true, nullptr, [&](int i, double v) { epi_d(i, v, pre_d(i)); });
      else if constexpr (kGlob)
        if (short_k)
          batch_rows_pg<kGSrc>(A.k_cptr, A.k_col, A.k_val, kr0, kr1, D.kc0, D.c0, xs, A, pre_d, epi_d);
        else
          batch_rows_p<kGSrc>(A.k_cptr, A.k_col, A.k_val, kr0, kr1, D.kc0, D.c0, xs, A, pre_d, epi_d);
      else
        batch_rows_p<kSrcSmemX>(A.k_cptr, A.k_col, A.k_val, kr0, kr1, D.kc0, D.c0, nullptr, A, pre_d, epi_d);
      T.sync();
      ++k;
      ++t;
      if (--until_check > 0 && k < A.max_iter) continue;
      until_check = A.check_every;
    }
    // ---- check
    if constexpr (kRes) {
      // running sums and K x back to global memory, where the check reads them
      for (int j = jc0 + tid; j < jc1; j += nt) A.sx[D.c0 + j] = sxv[j - jofs];
      for (int i = ir0 + tid; i < ir1; i += nt) {
        A.sy[D.r0 + i] = syv[i - iofs];
        A.kxp[D.r0 + i] = kxv[i - iofs];
      }
    }
    if constexpr (kCl) {
      // the averages are gathered from the owners' global running sums
      __threadfence();
      T.sync();
    } else if constexpr (kRes) {
      __syncthreads();
    }
    const double it = t > 0 ? 1.0 / (double)t : 0.0;
    Tmul(true, nullptr,
                                [&](int j, double s) { A.g[D.c0 + j] = s; });
    Kmul(false, A.sx + D.c0,
                                 [&](int i, double s) { A.kx_a[D.r0 + i] = s * it; });
    Tmul(false, A.sy + D.r0,
                                 [&](int j, double s) { A.g_a[D.c0 + j] = s * it; });
    __syncthreads();
    batch_kkt(A, D, t == 0, it, red, tot, ir0, ir1, jc0, jc1, part, flip, T, xs, ys);
    if (tid == 0) {
      S.k = k;
      S.t = t;
      S.inv_t = it;
      const long long nc = S.ncheck;
      const CheckRecord rec = decide_core(tot, &S, P, k >= A.max_iter,
                                          (T.rank == 0 && A.restarts) ? A.restarts + (size_t)b * A.restart_stride : nullptr);
      if (A.log != nullptr && T.rank == 0 && nc < P.log_cap) A.log[nc] = rec;
    }
    __syncthreads();
    if (S.done) break;
    const bool suspend = A.slice_iters > 0 && k - k_start >= A.slice_iters;
    if (S.restart_flag) {
      const bool avg = S.cand_avg;
      if (avg) {
        for (int j = xw0 + tid; j < xw1; j += nt) xs[j] = A.sx[D.c0 + j] * it;
        for (int i = yw0 + tid; i < yw1; i += nt) ys[i] = A.sy[D.r0 + i] * it;
      }
      T.sync();   // every replica is read before the owners clear the sums
      for (int j = jc0 + tid; j < jc1; j += nt) {
        A.xa[D.c0 + j] = xs[j];
        sxv[j - jofs] = 0.0;
      }
      for (int i = ir0 + tid; i < ir1; i += nt) {
        const int64_t gi = D.r0 + i;
        A.ya[gi] = ys[i];
        syv[i - iofs] = 0.0;
        if (avg) kxv[i - iofs] = A.kx_a[gi];
      }
      t = 0;
      __syncthreads();
    }
    if (suspend) break;
  }
  if (!S.done) {
    // ---- suspended by the iteration slice: the current point goes to xout / yout, the
    // running sums (written at this check), anchor and K x stay in global memory
    if constexpr (kRes) {
      // a restart at this check cleared the shared-memory sums and may have replaced K x
      for (int j = jc0 + tid; j < jc1; j += nt) A.sx[D.c0 + j] = sxv[j - jofs];
      for (int i = ir0 + tid; i < ir1; i += nt) {
        A.sy[D.r0 + i] = syv[i - iofs];
        A.kxp[D.r0 + i] = kxv[i - iofs];
      }
    }
    for (int j = jc0 + tid; j < jc1; j += nt) A.xout[D.c0 + j] = xs[j];
    for (int i = ir0 + tid; i < ir1; i += nt) A.yout[D.r0 + i] = ys[i];
    if (tid == 0 && T.rank == 0) {
      S.k = k;
      S.t = t;
      S.suspended = 1;
      A.st[b] = S;
    }
    T.sync();
    return;
  }
  // ---- returned point and state (the global sums were written at the last check)
  const bool avg = S.which == 1 && t > 0;
  const double it = t > 0 ? 1.0 / (double)t : 0.0;
  for (int j = jc0 + tid; j < jc1; j += nt) A.xout[D.c0 + j] = avg ? A.sx[D.c0 + j] * it : xs[j];
  for (int i = ir0 + tid; i < ir1; i += nt) A.yout[D.r0 + i] = avg ? A.sy[D.r0 + i] * it : ys[i];
  if (A.xcur != nullptr) {
    for (int j = jc0 + tid; j < jc1; j += nt) A.xcur[D.c0 + j] = xs[j];
    for (int i = ir0 + tid; i < ir1; i += nt) A.ycur[D.r0 + i] = ys[i];
  }
  if (tid == 0 && T.rank == 0) A.st[b] = S;
  T.sync();   // no CTA writes the next LP into a replica (or slice) that is still being read
}

// FP32 rows of chunks [c0, c1) (values A.k_val32 / t_val32 in global memory; gathers
// from the float replicas src); same order per row as batch_rows.
template <bool kGlobSrc, class F>
__device__ __forceinline__ void batch_rows32(const int32_t* __restrict__ cptr, const int32_t* __restrict__ col,
                                             const float* __restrict__ val, int c0, int c1, int cbase, int64_t base,
                                             const float* src, F epi) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int ch = c0 + wid; ch < c1; ch += nw) {
    const int s0 = cptr[ch], s1 = cptr[ch + 1];
    float acc = 0.0f;
    for (int s = s0; s < s1; s += kBB) {
      const int nb = min(kBB, s1 - s);
      float v[kBB], xv[kBB];
      int ci[kBB];
#pragma unroll
      for (int j = 0; j < kBB; ++j)
        if (j < nb) {
          v[j] = __ldcs(val + (size_t)(s + j) * 32 + lane);
          ci[j] = __ldcs(col + (size_t)(s + j) * 32 + lane) - (int)base;
        }
#pragma unroll
      for (int j = 0; j < kBB; ++j) xv[j] = j < nb ? (kGlobSrc ? __ldcg(src + ci[j]) : src[ci[j]]) : 0.0f;
#pragma unroll
      for (int j = 0; j < kBB; ++j)
        if (j < nb) acc = fmaf(v[j], xv[j], acc);
    }
    epi((ch - cbase) * 32 + lane, acc);
  }
}

// batch_rows32 with the epilogue operands and the next chunk's bounds loaded ahead.
template <bool kGlobSrc, class Pre, class F>
__device__ __forceinline__ void batch_rows32_p(const int32_t* __restrict__ cptr, const int32_t* __restrict__ col,
                                               const float* __restrict__ val, int c0, int c1, int cbase,
                                               int64_t base, const float* src, Pre pre, F epi) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  int ch = c0 + wid;
  int s0 = 0, s1 = 0;
  if (ch < c1) {
    s0 = cptr[ch];
    s1 = cptr[ch + 1];
  }
  for (; ch < c1; ch += nw) {
    const int row = (ch - cbase) * 32 + lane;
    const auto pv = pre(row);
    int n0 = 0, n1 = 0;
    if (ch + nw < c1) {
      n0 = cptr[ch + nw];
      n1 = cptr[ch + nw + 1];
    }
    if (PDLP_BATCH_L2PF && lane == 0 && n1 > n0) {
      const uint32_t ns = (uint32_t)min(n1 - n0, kPfSlots);
      l2_prefetch(val + (size_t)n0 * 32, ns * 128u);
      l2_prefetch(col + (size_t)n0 * 32, ns * 128u);
    }
    float acc = 0.0f;
    for (int s = s0; s < s1; s += kBB) {
      const int nb = min(kBB, s1 - s);
      float v[kBB], xv[kBB];
      int ci[kBB];
#pragma unroll
      for (int j = 0; j < kBB; ++j)
        if (j < nb) {
          v[j] = __ldcs(val + (size_t)(s + j) * 32 + lane);
          ci[j] = __ldcs(col + (size_t)(s + j) * 32 + lane) - (int)base;
        }
#pragma unroll
      for (int j = 0; j < kBB; ++j) xv[j] = j < nb ? (kGlobSrc ? __ldcg(src + ci[j]) : src[ci[j]]) : 0.0f;
#pragma unroll
      for (int j = 0; j < kBB; ++j)
        if (j < nb) acc = fmaf(v[j], xv[j], acc);
    }
    epi(row, acc, pv);
    s0 = n0;
    s1 = n1;
  }
}

// Mixed precision for a batch (the NEXT-1 split, one LP per team): FP32 iterations on
// float replicas, values and problem vectors, FP32 running sums over one check interval
// folded into the FP64 sums at every check; every check in FP64 (FP64 copy of the point
// in xout / yout, K x recomputed in FP64) with the restart rule of Section 2.  An LP
// whose FP64-measured error reaches A.switch_tol, or stops improving by 10 % for 16
// checks, is suspended with its FP64 state and finishes in FP64 (a resumed launch of
// k_batch_solve).  No resident slices.
template <bool kCl, bool kGlob>
__device__ void batch_solve_one32(const BatchArgs& A, int b, const Team<kCl>& T) {
  extern __shared__ double bsm[];
  const LpDesc& D0 = A.desc[b];
  // FP64 iterates (power iteration only) and FP32 iterates: shared-memory replicas over the
  // same space, or one copy each in global memory (kGlob)
  double* xs = kGlob ? A.xg + D0.c0 : bsm + A.xs_off;
  double* ys = kGlob ? A.yg + D0.r0 : bsm + A.ys_off;
  float* xf = kGlob ? A.xg32 + D0.c0 : reinterpret_cast<float*>(bsm + A.xs_off);
  float* yf = kGlob ? A.yg32 + D0.r0 : reinterpret_cast<float*>(bsm + A.ys_off);
  double* red = bsm + A.red_off;
  double* part = bsm + A.part_off;
  __shared__ DevState S;
  __shared__ double tot[NQ];
  __shared__ double scal[4];
  const LpDesc D = A.desc[b];
  const int n = D.n, m = D.m;
  const int tid = threadIdx.x, nt = blockDim.x;
  int flip = 0;
  const int kr0 = split_point(A.k_cptr, D.kc0, D.kc1, T.rank, T.size);
  const int kr1 = split_point(A.k_cptr, D.kc0, D.kc1, T.rank + 1, T.size);
  const int tr0 = split_point(A.t_cptr, D.tc0, D.tc1, T.rank, T.size);
  const int tr1 = split_point(A.t_cptr, D.tc0, D.tc1, T.rank + 1, T.size);
  const int ir0 = (kr0 - D.kc0) * 32, ir1 = (kr1 - D.kc0) * 32;
  const int jc0 = (tr0 - D.tc0) * 32, jc1 = (tr1 - D.tc0) * 32;
  const int mo1 = min(ir1, m), no1 = min(jc1, n);
  double* x64 = A.xout + D.c0;   // FP64 copy of the current point (all columns of the LP)
  double* y64 = A.yout + D.r0;
  const int xw0 = kGlob ? jc0 : 0, xw1 = kGlob ? jc1 : D.npad;
  const int yw0 = kGlob ? ir0 : 0, yw1 = kGlob ? ir1 : D.mpad;
  auto put = [&](auto* a, int i, auto v) {
    if constexpr (kGlob) a[i] = v;
    else T.put(a, i, v);
  };

  // ---- step size: power iteration on K'K in FP64 (as the FP64 solver)
  double eta = A.eta_fixed;
  if (!(eta > 0.0)) {
    const double v0 = 1.0 / sqrt((double)n);
    for (int j = xw0 + tid; j < xw1; j += nt) xs[j] = j < n ? v0 : 0.0;
    if constexpr (kGlob) T.sync();
    else __syncthreads();
    for (int it = 0; it < A.power_iters; ++it) {
      batch_rows<kGlob ? kSrcGlobal : kSrcSmemX, false>(A.k_cptr, A.k_col, A.k_val, kr0, kr1, D.kc0, D.c0, xs, A,
                                                         [&](int i, double s) { put(ys, i, s); });
      T.sync();
      batch_rows<kGlob ? kSrcGlobal : kSrcSmemY, false>(A.t_cptr, A.t_col, A.t_val, tr0, tr1, D.tc0, D.r0, ys, A,
                                                         [&](int j, double s) { A.g[D.c0 + j] = s; });
      __syncthreads();
      const double nw = team_norm(A.g + D.c0, jc0, jc1, red, part, flip, T);
      if (nw != 0.0)
        for (int j = jc0 + tid; j < jc1; j += nt) put(xs, j, A.g[D.c0 + j] / nw);
      T.sync();
    }
    batch_rows<kGlob ? kSrcGlobal : kSrcSmemX, false>(A.k_cptr, A.k_col, A.k_val, kr0, kr1, D.kc0, D.c0, xs, A,
                                                       [&](int i, double s) { put(ys, i, s); });
    T.sync();
    const double sn = m > 0 ? team_norm(ys, ir0, ir1, red, part, flip, T) : 0.0;
    eta = sn > 0.0 ? A.step_scale / sn : 1.0;
  }
  double omega = A.omega_fixed;
  {
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int j = jc0 + tid; j < no1; j += nt) {
      const double cj = A.c[D.c0 + j];
      const double cu = cj * A.invDc[D.c0 + j];
      a[0] = fma(cj, cj, a[0]);
      a[2] = fma(cu, cu, a[2]);
    }
    for (int i = ir0 + tid; i < mo1; i += nt) {
      const double qi = A.q[D.r0 + i];
      const double qu = qi * A.invDr[D.r0 + i];
      a[1] = fma(qi, qi, a[1]);
      a[3] = fma(qu, qu, a[3]);
    }
    team_sum<4>(a, red, part, flip, T);
    if (tid == 0) {
      const double cn = sqrt(red[0]), qn = sqrt(red[1]);
      scal[0] = (cn > 1e-10 && qn > 1e-10) ? cn / qn : 1.0;
      scal[1] = sqrt(red[2]);
      scal[2] = sqrt(red[3]);
    }
    __syncthreads();
    if (!(omega > 0.0)) omega = scal[0];
    if (A.omega0 != nullptr && A.omega0[b] > 0.0) omega = A.omega0[b];
  }
  DevParams P = A.P;
  P.cnorm = scal[1];
  P.qnorm = scal[2];

  // ---- initial point: FP64 copy (owners) and float replicas (every CTA), anchor, sums
  for (int j = xw0 + tid; j < xw1; j += nt) {
    const int64_t gj = D.c0 + j;
    const double x0 = j < n ? clamp_box(A.x0 ? A.x0[gj] : 0.0, A.l[gj], A.u[gj]) : 0.0;
    xf[j] = (float)x0;
    if (j >= jc0 && j < jc1) {
      x64[j] = x0;
      A.xa[gj] = x0;
      A.sx[gj] = 0.0;
      A.sx32[gj] = 0.0f;
    }
  }
  for (int i = yw0 + tid; i < yw1; i += nt) {
    const int64_t gi = D.r0 + i;
    double y0 = (A.y0 && i < m) ? A.y0[gi] : 0.0;
    if (i >= D.m1) y0 = max0(y0);
    yf[i] = (float)y0;
    if (i >= ir0 && i < ir1) {
      y64[i] = y0;
      A.ya[gi] = y0;
      A.sy[gi] = 0.0;
      A.sy32[gi] = 0.0f;
    }
  }
  __threadfence();
  T.sync();
  batch_rows<kSrcGlobal, false>(A.k_cptr, A.k_col, A.k_val, kr0, kr1, D.kc0, D.c0, x64, A, [&](int i, double s) {
    A.kxp[D.r0 + i] = s;
    A.kxp32[D.r0 + i] = (float)s;
  });
  batch_rows<kSrcGlobal, false>(A.t_cptr, A.t_col, A.t_val, tr0, tr1, D.tc0, D.r0, y64, A,
                                [&](int j, double s) { A.g[D.c0 + j] = s; });
  __syncthreads();
  if (tid == 0) {
    memset(&S, 0, sizeof(S));
    S.eta = eta;
    S.omega = omega;
    S.tau = eta / omega;
    S.sigma = eta * omega;
  }
  __syncthreads();
  batch_kkt(A, D, true, 0.0, red, tot, ir0, ir1, jc0, jc1, part, flip, T, x64, y64);
  if (tid == 0) {
    const double gap = tot[Q_QY_C] + tot[Q_LT_C] - tot[Q_CX_C];
    S.kkt_anchor = kkt_w(tot[Q_PRS_C], tot[Q_DRS_C], gap, S.omega);
    S.kkt_prev = __longlong_as_double(0x7FF0000000000000LL);
  }
  __syncthreads();

  // ---- FP32 iterations, FP64 checks
  long long k = 0, t = 0;
  int until_check = A.check_every;
  double best_err = __longlong_as_double(0x7FF0000000000000LL);
  int since_best = 0;
  bool to_fp64 = false;
  for (;;) {
    const bool at_limit = k >= A.max_iter;
    if (!at_limit) {
      const float tau = (float)S.tau, sigma = (float)S.sigma;
      struct PreP { float c, l, u, sx, x; };
      batch_rows32_p<kGlob>(
          A.t_cptr, A.t_col, A.t_val32, tr0, tr1, D.tc0, D.r0, yf,
          [&](int j) {
            const int64_t gj = D.c0 + j;
            return PreP{A.c32[gj], A.l32[gj], A.u32[gj], A.sx32[gj], xf[j]};
          },
          [&](int j, float gsum, const PreP& p) {
            float xn = fmaf(-tau, p.c - gsum, p.x);
            xn = fminf(fmaxf(xn, p.l), p.u);
            put(xf, j, xn);
            A.sx32[D.c0 + j] = p.sx + xn;
          });
      T.sync();
      struct PreD { float q, kx, y, sy; };
      batch_rows32_p<kGlob>(
          A.k_cptr, A.k_col, A.k_val32, kr0, kr1, D.kc0, D.c0, xf,
          [&](int i) {
            const int64_t gi = D.r0 + i;
            return PreD{A.q32[gi], A.kxp32[gi], yf[i], A.sy32[gi]};
          },
          [&](int i, float v, const PreD& p) {
            float yn = fmaf(sigma, fmaf(-2.0f, v, p.q + p.kx), p.y);
            if (i >= D.m1) yn = fmaxf(yn, 0.0f);
            put(yf, i, yn);
            const int64_t gi = D.r0 + i;
            A.sy32[gi] = p.sy + yn;
            A.kxp32[gi] = v;
          });
      T.sync();
      ++k;
      ++t;
      if (--until_check > 0 && k < A.max_iter) continue;
      until_check = A.check_every;
    }
    // ---- FP64 check: fold the interval sums, FP64 copy of the point, FP64 products
    for (int j = jc0 + tid; j < jc1; j += nt) {
      const int64_t gj = D.c0 + j;
      A.sx[gj] += (double)A.sx32[gj];
      A.sx32[gj] = 0.0f;
      x64[j] = (double)xf[j];
    }
    for (int i = ir0 + tid; i < ir1; i += nt) {
      const int64_t gi = D.r0 + i;
      A.sy[gi] += (double)A.sy32[gi];
      A.sy32[gi] = 0.0f;
      y64[i] = (double)yf[i];
    }
    __threadfence();
    T.sync();
    const double it = t > 0 ? 1.0 / (double)t : 0.0;
    batch_rows<kSrcGlobal, false>(A.k_cptr, A.k_col, A.k_val, kr0, kr1, D.kc0, D.c0, x64, A,
                                  [&](int i, double s) { A.kxp[D.r0 + i] = s; });
    batch_rows<kSrcGlobal, false>(A.t_cptr, A.t_col, A.t_val, tr0, tr1, D.tc0, D.r0, y64, A,
                                  [&](int j, double s) { A.g[D.c0 + j] = s; });
    batch_rows<kSrcGlobal, false>(A.k_cptr, A.k_col, A.k_val, kr0, kr1, D.kc0, D.c0, A.sx + D.c0, A,
                                  [&](int i, double s) { A.kx_a[D.r0 + i] = s * it; });
    batch_rows<kSrcGlobal, false>(A.t_cptr, A.t_col, A.t_val, tr0, tr1, D.tc0, D.r0, A.sy + D.r0, A,
                                  [&](int j, double s) { A.g_a[D.c0 + j] = s * it; });
    __syncthreads();
    batch_kkt(A, D, t == 0, it, red, tot, ir0, ir1, jc0, jc1, part, flip, T, x64, y64);
    if (tid == 0) {
      S.k = k;
      S.t = t;
      S.inv_t = it;
      decide_core(tot, &S, P, k >= A.max_iter,
                  (T.rank == 0 && A.restarts) ? A.restarts + (size_t)b * A.restart_stride : nullptr);
    }
    __syncthreads();
    if (S.done) break;
    // switch to FP64 iterations (the same test on every CTA: S is identical)
    const double e = S.last_err;
    if (e < 0.9 * best_err) {
      best_err = e;
      since_best = 0;
    } else {
      ++since_best;
    }
    to_fp64 = e <= A.switch_tol || since_best >= 16;
    if (S.restart_flag) {
      const bool avg = S.cand_avg;
      // every CTA refreshes its float replicas from the new FP64 point before the
      // owners overwrite the FP64 copy and clear the sums
      for (int j = xw0 + tid; j < xw1; j += nt) xf[j] = (float)(avg ? A.sx[D.c0 + j] * it : x64[j]);
      for (int i = yw0 + tid; i < yw1; i += nt) yf[i] = (float)(avg ? A.sy[D.r0 + i] * it : y64[i]);
      T.sync();
      for (int j = jc0 + tid; j < jc1; j += nt) {
        const int64_t gj = D.c0 + j;
        const double v = avg ? A.sx[gj] * it : x64[j];
        x64[j] = v;
        A.xa[gj] = v;
        A.sx[gj] = 0.0;
      }
      for (int i = ir0 + tid; i < ir1; i += nt) {
        const int64_t gi = D.r0 + i;
        const double v = avg ? A.sy[gi] * it : y64[i];
        y64[i] = v;
        A.ya[gi] = v;
        A.sy[gi] = 0.0;
        if (avg) A.kxp[gi] = A.kx_a[gi];
        A.kxp32[gi] = (float)A.kxp[gi];
      }
      t = 0;
      __syncthreads();
    } else {
      // K x of the FP32 iterations continues from its FP64 value
      for (int i = ir0 + tid; i < ir1; i += nt) A.kxp32[D.r0 + i] = (float)A.kxp[D.r0 + i];
      __syncthreads();
    }
    if (to_fp64) break;
  }
  if (!S.done) {
    // ---- to FP64: the point in xout / yout, FP64 sums, anchor and K x are all in place
    if (tid == 0 && T.rank == 0) {
      S.k = k;
      S.t = t;
      S.k32 = k;
      S.suspended = 1;
      A.st[b] = S;
    }
    T.sync();
    return;
  }
  const bool avg = S.which == 1 && t > 0;
  const double it = t > 0 ? 1.0 / (double)t : 0.0;
  for (int j = jc0 + tid; j < jc1; j += nt) A.xout[D.c0 + j] = avg ? A.sx[D.c0 + j] * it : x64[j];
  for (int i = ir0 + tid; i < ir1; i += nt) A.yout[D.r0 + i] = avg ? A.sy[D.r0 + i] * it : y64[i];
  if (tid == 0 && T.rank == 0) {
    S.k32 = k;
    A.st[b] = S;
  }
  T.sync();
}

template <bool kCl, bool kGlob>
__global__ void __launch_bounds__(256, (kGlob && !kCl) ? PDLP_BATCH32_GLOB_MIN_BLOCKS : PDLP_BATCH32_MIN_BLOCKS)
    k_batch_solve32(BatchArgs A) {
  __shared__ int lp;
  Team<kCl> T;
  T.init();
  const int teams = (int)gridDim.x / T.size;
  const int count = A.count;
  for (;;) {
    if (T.rank == 0 && threadIdx.x == 0) {
      const int v = atomicAdd(A.next, 1);
      if (v == count + teams - 1) *A.next = 0;
      for (int r = 0; r < T.size; ++r) *T.at(&lp, r) = v;
    }
    T.sync();
    const int v = lp;
    T.sync();
    if (v >= count) break;
    batch_solve_one32<kCl, kGlob>(A, A.order[v], T);
  }
}

// Persistent solver: teams draw LPs from the queue until it is empty.  The counter
// resets itself: the last of the failing draws (one per team) stores 0.
template <bool kCl, bool kRes, bool kGlob>
__global__ void __launch_bounds__(256, kCl ? (kGlob ? PDLP_BATCH_CL_GLOB_MIN_BLOCKS : 2) : (kGlob ? PDLP_BATCH_GLOB_MIN_BLOCKS : PDLP_BATCH_MIN_BLOCKS)) k_batch_solve(BatchArgs A) {
  __shared__ int lp;
  Team<kCl> T;
  T.init();
  const int teams = (int)gridDim.x / T.size;
  const int count = A.count;
  for (;;) {
    if (T.rank == 0 && threadIdx.x == 0) {
      const int v = atomicAdd(A.next, 1);
      if (v == count + teams - 1) *A.next = 0;
      for (int r = 0; r < T.size; ++r) *T.at(&lp, r) = v;
    }
    T.sync();
    const int v = lp;
    T.sync();
    if (v >= count) break;
    batch_solve_one<kCl, kRes, kGlob>(A, A.order[v], T);
  }
}

}  // namespace pdlp

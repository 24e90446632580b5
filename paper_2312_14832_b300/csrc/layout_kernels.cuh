// Device construction of the SELL-32 layouts of K and K' (the format is described in
// layout.h).  The host decides the row and column orders and the chunk lengths, which
// take O(m + n) work; everything that touches each nonzero runs here:
//   * a checked count of the entries of each column (k_check_count);
//   * the row of each entry (k_row_of);
//   * the entries of each column in increasing entry order, i.e. the CSC order of the
//     caller's CSR matrix, by a stable least-significant-digit radix sort of the entry
//     indices on their column (k_radix_hist, exclusive scan, k_radix_scatter);
//   * one thread per SELL slot and lane, gathering its column index and value
//     (k_fill_sell).
// The same layouts come out as from the host builder (build_sell): K rows keep the
// caller's entry order, K' rows list their entries by increasing row.
#pragma once
#include <cstdint>

#include "kernels.cuh"

namespace pdlp {

// Input-check flags.
enum : int { kBadCol = 1, kBadVal = 2 };

// Checks every entry of `count` LPs stored back to back (LP b: entries ent0[b] ..
// ent0[b+1] - 1, columns col0[b] .. col0[b+1] - 1 of the global numbering): a local
// column in [0, n_b) and a finite value.  Rewrites each column index as global and
// counts the entries of each global column; entries with a bad column are left alone.
__global__ void k_check_count(int32_t* __restrict__ col, const double* __restrict__ val, int64_t nnz,
                              const int64_t* __restrict__ ent0, const int64_t* __restrict__ col0, int64_t count,
                              int32_t* __restrict__ clen, int* __restrict__ flags) {
  int bad = 0;
  PDLP_GRID_STRIDE(k, nnz) {
    int64_t lo = 0, hi = count - 1;   // the LP of entry k: the last b with ent0[b] <= k
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (ent0[mid] <= k) lo = mid;
      else hi = mid - 1;
    }
    const int64_t c0 = col0[lo], nb = col0[lo + 1] - c0;
    const int32_t j = col[k];
    if (j < 0 || j >= nb) {
      bad |= kBadCol;
    } else {
      col[k] = (int32_t)(c0 + j);
      atomicAdd(&clen[c0 + j], 1);
    }
    if (!isfinite(val[k])) bad |= kBadVal;
  }
  if (bad) atomicOr(flags, bad);
}

// rowof[k] = i for every entry k of row i (one warp per row).
__global__ void k_row_of(const int64_t* __restrict__ rp, int64_t m, int32_t* __restrict__ rowof) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = w0; i < m; i += nw)
    for (int64_t k = rp[i] + lane; k < rp[i + 1]; k += 32) rowof[k] = (int32_t)i;
}

// ---- exclusive prefix sums of int32 arrays (totals below 2^31)

constexpr int kScanThreads = 1024, kScanItems = 4, kScanTile = kScanThreads * kScanItems;

// Exclusive scan of each tile of kScanTile elements in place; the tile's total goes to
// sums[tile].
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(int32_t* __restrict__ a, int64_t n,
                                                             int32_t* __restrict__ sums) {
  __shared__ int32_t wsum[32];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int64_t i0 = (int64_t)blockIdx.x * kScanTile + (int64_t)tid * kScanItems;
  int32_t v[kScanItems], s = 0;
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    v[q] = i0 + q < n ? a[i0 + q] : 0;
    s += v[q];
  }
  int32_t x = s;   // inclusive scan of the thread sums within the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    int32_t z = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, z, o);
      if (lane >= o) z += y;
    }
    wsum[lane] = z;
  }
  __syncthreads();
  int32_t ex = x - s + (w > 0 ? wsum[w - 1] : 0);
#pragma unroll
  for (int q = 0; q < kScanItems; ++q) {
    if (i0 + q < n) a[i0 + q] = ex;
    ex += v[q];
  }
  if (tid == kScanThreads - 1) sums[blockIdx.x] = ex;
}

// Adds each tile's offset (the exclusive scan of the tile totals).
__global__ void k_scan_add(int32_t* __restrict__ a, int64_t n, const int32_t* __restrict__ sums) {
  PDLP_GRID_STRIDE(i, n) a[i] += sums[i / kScanTile];
}

// ---- stable LSD radix sort of (key, value) int32 pairs, 8 bits per pass

constexpr int kRadixThreads = 256, kRadixItems = 16, kRadixTile = kRadixThreads * kRadixItems;

// hist[d * tiles + b] = number of keys of tile b whose digit (key >> shift) & 255 is d.
__global__ void __launch_bounds__(kRadixThreads) k_radix_hist(const int32_t* __restrict__ key, int64_t count,
                                                              int shift, int32_t* __restrict__ hist, int64_t tiles) {
  __shared__ int32_t hs[256];
  hs[threadIdx.x] = 0;
  __syncthreads();
  const int64_t t0 = (int64_t)blockIdx.x * kRadixTile;
  for (int r = 0; r < kRadixItems; ++r) {
    const int64_t k = t0 + (int64_t)r * kRadixThreads + threadIdx.x;
    if (k < count) atomicAdd(&hs[(key[k] >> shift) & 255], 1);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = hs[threadIdx.x];
}

// Moves each pair of tile b to off[d * tiles + b] (the exclusive scan of hist) plus its
// rank among the earlier pairs of the tile with the same digit.  The tile is taken in
// rounds of 256 consecutive pairs; within a round a warp ranks its lanes with
// __match_any_sync and the warps' counts are prefixed per digit, so pairs with equal
// digits keep their order.  val_in == nullptr stands for the values 0, 1, 2, ...
__global__ void __launch_bounds__(kRadixThreads) k_radix_scatter(
    const int32_t* __restrict__ key_in, const int32_t* __restrict__ val_in, int64_t count, int shift,
    const int32_t* __restrict__ off, int64_t tiles, int32_t* __restrict__ key_out, int32_t* __restrict__ val_out) {
  __shared__ int32_t base[256];
  __shared__ int32_t wc[kRadixThreads / 32][256];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  base[tid] = off[(int64_t)tid * tiles + blockIdx.x];
#pragma unroll
  for (int q = 0; q < kRadixThreads / 32; ++q) wc[q][tid] = 0;
  __syncthreads();
  const int64_t t0 = (int64_t)blockIdx.x * kRadixTile;
  for (int r = 0; r < kRadixItems; ++r) {
    const int64_t k = t0 + (int64_t)r * kRadixThreads + tid;
    const bool ok = k < count;
    int32_t kk = 0, vv = 0, d = -1;
    if (ok) {
      kk = key_in[k];
      vv = val_in ? val_in[k] : (int32_t)k;
      d = (kk >> shift) & 255;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (ok && lane == __ffs(peers) - 1) wc[w][d] = __popc(peers);
    __syncthreads();
    int32_t acc = 0;   // this thread's digit: exclusive prefix over the warps
#pragma unroll
    for (int q = 0; q < kRadixThreads / 32; ++q) {
      const int32_t c = wc[q][tid];
      wc[q][tid] = acc;
      acc += c;
    }
    __syncthreads();
    if (ok) {
      const int32_t pos = base[d] + wc[w][d] + rank;
      key_out[pos] = kk;
      val_out[pos] = vv;
    }
    __syncthreads();
    base[tid] += acc;
#pragma unroll
    for (int q = 0; q < kRadixThreads / 32; ++q) wc[q][tid] = 0;
    __syncthreads();
  }
}

// ---- SELL fill

// One thread per (slot, lane) of a SELL-32 layout with chunk_ptr cptr (nchunks + 1
// entries, each chunk at least one slot).  Slot s lies in the chunk ch with
// cptr[ch] <= s < cptr[ch + 1]; its row is p = 32 ch + lane, or, in a wide chunk, the
// chunk's first row with entry (s - cptr[ch]) * 32 + lane.  Row p is the source row
// r = perm[p] (-1: padding) whose entries are q = order[t] (order == nullptr: q = t) for
// t in [ptr[r], ptr[r + 1]); an entry's output column is kmap[key[q]] and its value
// val[q].  Padding slots take value 0 and the column of the row's first entry, or for
// an empty row pad[ch] (the first internal column of the chunk's LP), as in build_sell.
template <class PT>
__global__ void k_fill_sell(const int32_t* __restrict__ cptr, int64_t nchunks, const uint8_t* __restrict__ wide,
                            int64_t total, const int32_t* __restrict__ perm, const PT* __restrict__ ptr,
                            const int32_t* __restrict__ order, const int32_t* __restrict__ key,
                            const int32_t* __restrict__ kmap, const double* __restrict__ val,
                            const int32_t* __restrict__ pad, int32_t* __restrict__ out_col,
                            double* __restrict__ out_val) {
  PDLP_GRID_STRIDE(e, total) {
    const int64_t s = e >> 5;
    const int lane = (int)(e & 31);
    int64_t lo = 0, hi = nchunks - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi + 1) >> 1;
      if (cptr[mid] <= s) lo = mid;
      else hi = mid - 1;
    }
    const bool wd = wide != nullptr && wide[lo] != 0;
    const int64_t p = lo * 32 + (wd ? 0 : lane);
    const int64_t off = wd ? (s - cptr[lo]) * 32 + lane : s - cptr[lo];
    const int32_t r = perm[p];
    int64_t st = 0, len = 0;
    if (r >= 0) {
      st = (int64_t)ptr[r];
      len = (int64_t)ptr[r + 1] - st;
    }
    if (off < len) {
      const int64_t q = order ? (int64_t)order[st + off] : st + off;
      out_col[e] = kmap[key[q]];
      out_val[e] = val[q];
    } else {
      int32_t c = pad[lo];
      if (len > 0) c = kmap[key[order ? (int64_t)order[st] : st]];
      out_col[e] = c;
      out_val[e] = 0.0;
    }
  }
}

}  // namespace pdlp

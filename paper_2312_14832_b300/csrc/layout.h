// The SELL-32 layout of K and K' and its host-side parts: the chunk shapes (sell_shape),
// the warp-task plan (plan_tasks) and the complete host builder (build_sell), which the
// device builder of layout_kernels.cuh reproduces and the tests compare against.
//
// Rows are renumbered in order of decreasing length (equality rows keep the
// first m1 positions, so the dual sign projection stays "row >= m1"), columns
// likewise.  Each matrix is stored "SELL-32": 32 consecutive rows form a chunk,
// and slot k of a chunk holds entry k of each of its 32 rows side by side, so a
// warp reads one slot with one fully coalesced 256-byte load and every lane owns
// one row.  A chunk is as long as its longest row (at least one slot); shorter
// rows are padded with zero values.  Work is cut into warp tasks of about
// `tile_slots` slots: short chunks are packed whole into a task (at most
// `tile_chunks` of them, so that a warp never runs a long serial chain of tiny
// chunks), a chunk longer
// than tile_slots is split into pieces whose partial sums are combined, in piece
// order, by the warp that finishes last.
//
// A "wide" row (one far longer than the rows next to it in length order, such as a
// dense row) gets a chunk of its own, whose other 31 rows are empty padding rows: its
// entries are spread over the 32 lanes (entry k in slot k / 32, lane k % 32), and the
// lanes' partial sums are combined by a fixed warp reduction.  So the row costs its own
// length / 32 slots instead of its length times 32.
#pragma once
#include <algorithm>
#include <cstdint>
#include <thread>
#include <vector>

namespace pdlp {

// Runs f(begin, end) over [0, n) cut into contiguous ranges, one per host thread (up to
// the hardware's count, and only as many as leave min_per_thread items each).  Every
// index is handled by exactly one call; f must not throw (report failures through
// per-range results instead).
template <class F>
void parallel_ranges(int64_t n, F f, int64_t min_per_thread = (int64_t)1 << 16) {
  if (n <= 0) return;
  int64_t t = (int64_t)std::max(1u, std::thread::hardware_concurrency());
  t = std::min<int64_t>(t, 32);
  t = std::max<int64_t>(1, std::min<int64_t>(t, n / std::max<int64_t>(1, min_per_thread)));
  if (t == 1) {
    f((int64_t)0, n);
    return;
  }
  std::vector<std::thread> th;
  th.reserve((size_t)t);
  for (int64_t i = 0; i < t; ++i) th.emplace_back([&, i]() { f(n * i / t, n * (i + 1) / t); });
  for (auto& x : th) x.join();
}

struct SellTask {
  int32_t s0, s1;   // slot range [s0, s1) of this warp task
  int32_t chunk;    // first chunk the task touches
  int32_t t0;       // split chunk: index of its first piece task; else -1
  int32_t np;       // split chunk: number of pieces; else 0
  int32_t nc;       // chunks the task covers (1 for a split piece)
  int32_t wide;     // 1: the task's chunk holds one wide row spread over the lanes
  int32_t pad;
};

struct SellHost {
  int64_t rows = 0;       // logical rows
  int64_t rows_pad = 0;   // rows rounded up to a multiple of 32 (at least 32)
  int64_t nchunks = 0;
  std::vector<int32_t> chunk_ptr;  // nchunks + 1, in slots
  std::vector<int32_t> col;        // slots * 32, internal column index
  std::vector<int32_t> src;        // slots * 32, position in the input CSR (-1 in padding)
  std::vector<uint8_t> wide;       // nchunks: 1 when the chunk holds one wide row
  int64_t slots() const { return chunk_ptr.empty() ? 0 : chunk_ptr.back(); }
};

struct TaskPlan {
  std::vector<SellTask> tasks;
  int64_t split_chunks = 0;
};

// Permutation by decreasing length (stable) of the indices [lo, hi), written to perm[lo..hi).
void sort_by_length_desc(const std::vector<int32_t>& len, int64_t lo, int64_t hi,
                         std::vector<int32_t>& perm);

// The shape of the SELL-32 layout of a matrix whose internal row p (0 <= p < rows) has
// elen[p] entries: chunk_ptr and the wide flags, no entry arrays.  wide_row (optional,
// per row): rows stored spread over their chunk's lanes; such a row is the first of its
// chunk and the other 31 rows of the chunk are empty.
SellHost sell_shape(int64_t rows, const std::vector<int32_t>& elen, const std::vector<uint8_t>* wide_row = nullptr);

// sell_shape plus the entry arrays: row p has the entries estart[p] .. estart[p] +
// elen[p] - 1 of ecol / esrc.  Padding slots take the column of the row's first entry,
// or pad_col for an empty row.
SellHost build_sell(int64_t rows, const std::vector<int64_t>& estart,
                    const std::vector<int32_t>& elen, const std::vector<int32_t>& ecol,
                    const std::vector<int32_t>& esrc, int32_t pad_col = 0,
                    const std::vector<uint8_t>* wide_row = nullptr);

// Appends the chunks of S after those of G (block-diagonal concatenation; the column
// indices of S must already be in G's numbering).
void append_sell(SellHost& G, const SellHost& S);

// Packs whole chunks into tasks of at most tile_slots slots and at most tile_chunks
// (<= 32) chunks; chunks longer than tile_slots become split pieces; a wide chunk is
// never packed with another.
TaskPlan plan_tasks(const SellHost& S, int32_t tile_slots, int32_t tile_chunks);

}  // namespace pdlp

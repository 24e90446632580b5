"""Host-side layout logic (csrc/layout.cpp) on the CPU: the length sort, the SELL-32
shape, the host builder (the reference the device builder is compared against on the
GPU) and the warp-task plan, compiled with g++ and driven on seeded random matrices
with empty, short, long and wide rows.  The driver checks, and reports the first
failure of:

  * sort_by_length_desc: a permutation of [lo, hi), lengths non-increasing, equal
    lengths in increasing index;
  * sell_shape: the same chunk pointers as build_sell; a chunk as long as its longest
    row (at least one slot), a wide chunk ceil(length / 32) slots;
  * build_sell: every entry in exactly one slot, entry k of a row in slot k and the
    row's lane (a wide row: slot k / 32, lane k % 32) with its column; padding slots
    with source -1 and the row's first column (pad_col for an empty row);
  * plan_tasks: the tasks tile the slots in order; a packed task holds whole chunks,
    at most tile_chunks of them and at most tile_slots slots, and never a wide chunk
    beside another; a split chunk's pieces are consecutive, cover it, and name their
    first piece and count.
"""
import os
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2312_14832_b300", "csrc")

DRIVER = r"""
#include "layout.h"
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>
using namespace pdlp;

static unsigned long long st;
static unsigned rnd() { st = st * 6364136223846793005ULL + 1442695040888963407ULL; return (unsigned)(st >> 33); }
#define FAIL(...) do { std::printf(__VA_ARGS__); std::printf("\n"); return 1; } while (0)

int main(int argc, char** argv) {
  st = std::strtoull(argv[1], nullptr, 10) * 2654435761ULL + 7;
  const int rows = std::atoi(argv[2]), ncol = std::atoi(argv[3]), nwide = std::atoi(argv[4]);
  // row lengths: a mixture of empty, short, chunk-boundary and long rows
  std::vector<int32_t> len(rows);
  for (int r = 0; r < rows; ++r) {
    const unsigned u = rnd() % 100;
    len[r] = u < 10 ? 0 : u < 60 ? (int)(rnd() % 8) : u < 85 ? 30 + (int)(rnd() % 5) : u < 97 ? (int)(rnd() % 200) : (int)(rnd() % 1500);
  }
  for (int w = 0; w < nwide && w < rows; ++w) len[w] = 3000 + (int)(rnd() % 2000);   // wide rows
  std::vector<int32_t> perm(rows);
  sort_by_length_desc(len, 0, rows, perm);
  {
    std::vector<char> seen(rows, 0);
    for (int p = 0; p < rows; ++p) {
      const int r = perm[p];
      if (r < 0 || r >= rows || seen[r]) FAIL("sort: not a permutation at %d", p);
      seen[r] = 1;
      if (p > 0) {
        const int q = perm[p - 1];
        if (len[q] < len[r]) FAIL("sort: lengths increase at %d", p);
        if (len[q] == len[r] && q > r) FAIL("sort: not stable at %d", p);
      }
    }
  }
  // internal rows: the wide rows first, each at a chunk start with 31 empty rows after
  // it, then the others in sorted order
  std::vector<int32_t> ord;
  std::vector<uint8_t> wflag;
  for (int p = 0; p < rows; ++p) {
    const int r = perm[p];
    if (r < nwide) {
      while (ord.size() % 32) { ord.push_back(-1); wflag.push_back(0); }
      ord.push_back(r); wflag.push_back(1);
      for (int k = 0; k < 31; ++k) { ord.push_back(-1); wflag.push_back(0); }
    }
  }
  for (int p = 0; p < rows; ++p)
    if (perm[p] >= nwide) { ord.push_back(perm[p]); wflag.push_back(0); }
  const int64_t R = (int64_t)ord.size();
  wflag.resize((size_t)((R + 31) / 32 * 32 + 32), 0);
  // entries: row r's entries are consecutive in the entry arrays
  std::vector<int64_t> rstart(rows + 1, 0);
  for (int r = 0; r < rows; ++r) rstart[r + 1] = rstart[r] + len[r];
  const int64_t nnz = rstart[rows];
  std::vector<int32_t> ecol((size_t)nnz), esrc((size_t)nnz);
  for (int64_t k = 0; k < nnz; ++k) { ecol[k] = (int32_t)(rnd() % ncol); esrc[k] = (int32_t)(1000000 + k); }
  std::vector<int64_t> estart((size_t)R);
  std::vector<int32_t> elen((size_t)R);
  for (int64_t p = 0; p < R; ++p) {
    estart[p] = ord[p] >= 0 ? rstart[ord[p]] : 0;
    elen[p] = ord[p] >= 0 ? len[ord[p]] : 0;
  }
  const int32_t pad_col = 77;
  SellHost S = build_sell(R, estart, elen, ecol, esrc, pad_col, &wflag);
  SellHost Z = sell_shape(R, elen, &wflag);
  if (Z.chunk_ptr != S.chunk_ptr || Z.wide != S.wide) FAIL("shape: differs from build_sell");
  if (S.rows_pad % 32 || S.rows_pad < R || S.nchunks * 32 != S.rows_pad) FAIL("shape: padding");
  std::vector<int> hit((size_t)nnz, 0);
  for (int64_t ch = 0; ch < S.nchunks; ++ch) {
    const int64_t base = S.chunk_ptr[ch], L = S.chunk_ptr[ch + 1] - base;
    const bool wd = S.wide[ch] != 0;
    int64_t want = 1;
    if (wd) want = std::max<int64_t>(1, (elen[ch * 32] + 31) / 32);
    else for (int64_t r = ch * 32; r < std::min<int64_t>(R, ch * 32 + 32); ++r) want = std::max<int64_t>(want, elen[r]);
    if (L != want) FAIL("shape: chunk %lld has %lld slots, wants %lld", (long long)ch, (long long)L, (long long)want);
    for (int64_t k = 0; k < L; ++k)
      for (int lane = 0; lane < 32; ++lane) {
        const int64_t e = (base + k) * 32 + lane;
        const int64_t r = wd ? ch * 32 : ch * 32 + lane;
        const int64_t idx = wd ? k * 32 + lane : k;   // entry index within the row
        const int64_t rl = r < R ? elen[r] : 0;
        if (idx < rl) {
          const int64_t q = estart[r] + idx;
          if (S.src[e] != esrc[q] || S.col[e] != ecol[q]) FAIL("fill: slot %lld lane %d", (long long)(base + k), lane);
          hit[q]++;
        } else {
          const int32_t pc = rl > 0 ? ecol[estart[r]] : pad_col;
          if (S.src[e] != -1 || S.col[e] != pc) FAIL("fill: padding slot %lld lane %d", (long long)(base + k), lane);
        }
      }
  }
  for (int64_t q = 0; q < nnz; ++q)
    if (hit[q] != 1) FAIL("fill: entry %lld placed %d times", (long long)q, hit[q]);
  const int tiles[][2] = {{32, 4}, {64, 1}, {8, 32}, {1, 1}};
  for (const auto& tc : tiles) {
    const int Q = tc[0], C = tc[1];
    TaskPlan P = plan_tasks(S, Q, C);
    int32_t s = 0;
    int64_t split = 0;
    for (size_t t = 0; t < P.tasks.size(); ++t) {
      const SellTask& T = P.tasks[t];
      if (T.s0 != s || T.s1 <= T.s0) FAIL("plan %d/%d: task %zu does not continue the slots", Q, C, t);
      const int32_t clen = S.chunk_ptr[T.chunk + 1] - S.chunk_ptr[T.chunk];
      if (T.np > 0) {
        if (T.t0 > (int)t || (int)t >= T.t0 + T.np || T.nc != 1) FAIL("plan %d/%d: split task %zu", Q, C, t);
        if ((int)t == T.t0) {
          ++split;
          if (T.s0 != S.chunk_ptr[T.chunk] || clen <= Q) FAIL("plan %d/%d: split chunk %d", Q, C, T.chunk);
          const SellTask& last = P.tasks[T.t0 + T.np - 1];
          if (last.chunk != T.chunk || last.s1 != S.chunk_ptr[T.chunk + 1]) FAIL("plan %d/%d: pieces of %d", Q, C, T.chunk);
        }
        if ((T.wide != 0) != (S.wide[T.chunk] != 0)) FAIL("plan %d/%d: wide flag of task %zu", Q, C, t);
      } else {
        if (T.t0 != -1 || T.nc < 1 || T.nc > C) FAIL("plan %d/%d: packed task %zu holds %d chunks", Q, C, t, T.nc);
        if (T.s0 != S.chunk_ptr[T.chunk] || T.s1 != S.chunk_ptr[T.chunk + T.nc]) FAIL("plan %d/%d: task %zu cuts a chunk", Q, C, t);
        if (T.s1 - T.s0 > Q && !(T.nc == 1 && S.wide[T.chunk])) FAIL("plan %d/%d: task %zu too long", Q, C, t);
        for (int c = T.chunk; c < T.chunk + T.nc; ++c)
          if (S.wide[c] && T.nc != 1) FAIL("plan %d/%d: wide chunk %d packed with others", Q, C, c);
      }
      s = T.s1;
    }
    if (s != S.chunk_ptr[S.nchunks]) FAIL("plan %d/%d: tasks end at slot %d of %d", Q, C, s, S.chunk_ptr[S.nchunks]);
    if (split != P.split_chunks) FAIL("plan %d/%d: split count", Q, C);
  }
  std::printf("ok rows=%d nnz=%lld chunks=%lld slots=%d\n", rows, (long long)nnz, (long long)S.nchunks,
              S.chunk_ptr[S.nchunks]);
  return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    d = tmp_path_factory.mktemp("layout")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    exe = d / "driver"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-pthread", "-I", CSRC, str(src),
                           os.path.join(CSRC, "layout.cpp"), "-o", str(exe)])
    return str(exe)


@pytest.mark.parametrize("seed,rows,ncol,nwide", [
    (1, 1, 5, 0), (2, 31, 40, 0), (3, 33, 100, 0), (4, 1000, 5000, 0), (5, 5000, 300, 3),
    (6, 777, 50000, 1), (7, 20000, 20000, 0), (8, 64, 10, 2)])
def test_host_layout_invariants(driver, seed, rows, ncol, nwide):
    out = subprocess.run([driver, str(seed), str(rows), str(ncol), str(nwide)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout + out.stderr

// Host-side construction of the SELL-32 layout and the warp task plan (see layout.h).
#include "layout.h"

#include <algorithm>

namespace pdlp {

void sort_by_length_desc(const std::vector<int32_t>& len, int64_t lo, int64_t hi,
                         std::vector<int32_t>& perm) {
  if (hi <= lo) return;
  int64_t maxlen = 0;
  for (int64_t i = lo; i < hi; ++i) maxlen = std::max<int64_t>(maxlen, len[(size_t)i]);
  // counting sort on length, descending, stable in the original index
  std::vector<int64_t> cnt((size_t)maxlen + 2, 0);
  for (int64_t i = lo; i < hi; ++i) cnt[(size_t)(maxlen - len[(size_t)i])]++;
  int64_t acc = lo;
  for (size_t b = 0; b < cnt.size(); ++b) {
    int64_t c = cnt[b];
    cnt[b] = acc;
    acc += c;
  }
  for (int64_t i = lo; i < hi; ++i) perm[(size_t)cnt[(size_t)(maxlen - len[(size_t)i])]++] = (int32_t)i;
}

SellHost sell_shape(int64_t rows, const std::vector<int32_t>& elen, const std::vector<uint8_t>* wide_row) {
  SellHost S;
  S.rows = rows;
  S.rows_pad = std::max<int64_t>(32, (rows + 31) / 32 * 32);
  S.nchunks = S.rows_pad / 32;
  S.chunk_ptr.assign((size_t)S.nchunks + 1, 0);
  S.wide.assign((size_t)S.nchunks, 0);
  for (int64_t ch = 0; ch < S.nchunks; ++ch) {
    int64_t L = 1;
    if (wide_row && ch * 32 < rows && (*wide_row)[(size_t)(ch * 32)]) {
      S.wide[(size_t)ch] = 1;
      L = std::max<int64_t>(1, ((int64_t)elen[(size_t)(ch * 32)] + 31) / 32);
    } else {
      for (int64_t r = ch * 32; r < std::min(rows, ch * 32 + 32); ++r) L = std::max<int64_t>(L, elen[(size_t)r]);
    }
    S.chunk_ptr[(size_t)ch + 1] = S.chunk_ptr[(size_t)ch] + (int32_t)L;
  }
  return S;
}

SellHost build_sell(int64_t rows, const std::vector<int64_t>& estart,
                    const std::vector<int32_t>& elen, const std::vector<int32_t>& ecol,
                    const std::vector<int32_t>& esrc, int32_t pad_col, const std::vector<uint8_t>* wide_row) {
  SellHost S = sell_shape(rows, elen, wide_row);
  size_t total = (size_t)S.chunk_ptr.back() * 32;
  S.col.resize(total);
  S.src.resize(total);
  // chunks are independent: each writes its own slots (entries, then padding)
  parallel_ranges(S.nchunks, [&](int64_t ch0, int64_t ch1) {
    for (int64_t ch = ch0; ch < ch1; ++ch) {
      const int64_t base = S.chunk_ptr[(size_t)ch];
      const int64_t clen = S.chunk_ptr[(size_t)ch + 1] - base;
      if (S.wide[(size_t)ch]) {
        // entry k of the row in slot k / 32, lane k % 32; padding gathers its first column
        const int64_t r = ch * 32, st = estart[(size_t)r], L = elen[(size_t)r];
        for (int64_t k = 0; k < clen * 32; ++k) {
          const size_t e = (size_t)base * 32 + (size_t)k;
          if (k < L) {
            S.col[e] = ecol[(size_t)(st + k)];
            S.src[e] = esrc[(size_t)(st + k)];
          } else {
            S.col[e] = L > 0 ? ecol[(size_t)st] : pad_col;
            S.src[e] = -1;
          }
        }
        continue;
      }
      for (int64_t lane = 0; lane < 32; ++lane) {
        const int64_t r = ch * 32 + lane;
        const int64_t st = r < rows ? estart[(size_t)r] : 0, L = r < rows ? elen[(size_t)r] : 0;
        for (int64_t k = 0; k < L; ++k) {
          const size_t e = (size_t)(base + k) * 32 + (size_t)lane;
          S.col[e] = ecol[(size_t)(st + k)];
          S.src[e] = esrc[(size_t)(st + k)];
        }
        // padding slots gather the row's own first column (already in cache), value 0
        const int32_t pc = L > 0 ? ecol[(size_t)st] : pad_col;
        for (int64_t k = L; k < clen; ++k) {
          const size_t e = (size_t)(base + k) * 32 + (size_t)lane;
          S.col[e] = pc;
          S.src[e] = -1;
        }
      }
    }
  }, 256);
  return S;
}

void append_sell(SellHost& G, const SellHost& S) {
  if (G.chunk_ptr.empty()) G.chunk_ptr.push_back(0);
  const int32_t base = G.chunk_ptr.back();
  for (int64_t ch = 0; ch < S.nchunks; ++ch) G.chunk_ptr.push_back(base + S.chunk_ptr[(size_t)ch + 1]);
  G.col.insert(G.col.end(), S.col.begin(), S.col.end());
  G.src.insert(G.src.end(), S.src.begin(), S.src.end());
  G.wide.insert(G.wide.end(), S.wide.begin(), S.wide.end());
  G.rows += S.rows_pad;
  G.rows_pad = G.rows;
  G.nchunks += S.nchunks;
}

TaskPlan plan_tasks(const SellHost& S, int32_t Q, int32_t C) {
  TaskPlan P;
  if (Q < 1) Q = 1;
  if (C < 1) C = 1;
  if (C > 32) C = 32;
  int64_t c = 0;
  auto is_wide = [&](int64_t ch) { return !S.wide.empty() && S.wide[(size_t)ch] != 0; };
  while (c < S.nchunks) {
    int32_t base = S.chunk_ptr[(size_t)c];
    int32_t len = S.chunk_ptr[(size_t)c + 1] - base;
    if (is_wide(c) && len <= Q) {
      SellTask T{};
      T.s0 = base;
      T.s1 = base + len;
      T.chunk = (int32_t)c;
      T.t0 = -1;
      T.np = 0;
      T.nc = 1;
      T.wide = 1;
      P.tasks.push_back(T);
      ++c;
    } else if (len > Q) {
      int32_t np = (len + Q - 1) / Q;
      int32_t t0 = (int32_t)P.tasks.size();
      for (int32_t i = 0; i < np; ++i) {
        SellTask T{};
        T.s0 = base + (int32_t)(((int64_t)len * i) / np);
        T.s1 = base + (int32_t)(((int64_t)len * (i + 1)) / np);
        T.chunk = (int32_t)c;
        T.t0 = t0;
        T.np = np;
        T.nc = 1;
        T.wide = is_wide(c) ? 1 : 0;
        P.tasks.push_back(T);
      }
      P.split_chunks++;
      ++c;
    } else {
      SellTask T{};
      T.s0 = base;
      T.chunk = (int32_t)c;
      T.t0 = -1;
      T.np = 0;
      int32_t tot = 0, nc = 0;
      while (c < S.nchunks && nc < C) {
        int32_t l = S.chunk_ptr[(size_t)c + 1] - S.chunk_ptr[(size_t)c];
        if (l > Q || tot + l > Q || is_wide(c)) break;
        tot += l;
        ++nc;
        ++c;
      }
      T.s1 = S.chunk_ptr[(size_t)c];
      T.nc = nc;
      P.tasks.push_back(T);
    }
  }
  return P;
}

}  // namespace pdlp

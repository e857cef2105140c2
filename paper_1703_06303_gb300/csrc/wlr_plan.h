// Host-side launch planning of the sWLR kernels (no CUDA calls): the row chunks of the
// split-m Gram products, whose chunk partials are summed afterwards in a fixed order.
#pragma once

#include <algorithm>
#include <climits>
#include <cstddef>
#include <cstdint>
#include <utility>
#include <vector>

namespace wlr {

inline int cdiv(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

struct Chunk {
  int nch, rows;   // number of row chunks, rows per chunk (a multiple of 32)
};

// row chunks for a split-m Gram with `tiles` output tiles: about `target` blocks in
// all, at most 128 chunks (each chunk is a partial the consumer sums).
inline Chunk chunking(int m, size_t tiles, int target = 160) {
  int nch = std::max<int>(1, (int)((target + tiles - 1) / std::max<size_t>(tiles, 1)));
  nch = std::min(nch, 128);
  int rows = cdiv(m, nch);
  rows = std::max(32, ((rows + 31) / 32) * 32);
  nch = std::max(1, cdiv(m, rows));
  return {nch, rows};
}
// row chunks for a kernel with `tiles` independent output tiles whose CTAs occupy `slots`
// places on the GPU at a time (SMs x CTAs per SM).  The time of the busiest SM is about
// waves x (rows per chunk + a pipeline fill of 128 rows); the fewest chunks within 3% of
// the best such time are taken (fewer partial sums to add afterwards).
inline Chunk chunking_waves(int m, int tiles, int slots) {
  slots = std::max(slots, 1);
  const int nmax = std::max(1, std::min(128, cdiv(m, 32)));
  std::vector<std::pair<Chunk, int64_t>> cand;
  int64_t best_cost = INT64_MAX;
  for (int n = 1; n <= nmax; ++n) {
    const int rows = std::max(32, ((cdiv(m, n) + 31) / 32) * 32);
    const int nn = cdiv(m, rows);
    const int64_t cost = (int64_t)cdiv(tiles * nn, slots) * (rows + 128);
    cand.push_back({Chunk{nn, rows}, cost});
    best_cost = std::min(best_cost, cost);
  }
  Chunk pick{0, 0};
  for (const auto& c : cand)
    if (c.second == best_cost) {
      pick = c.first;
      break;
    }
  for (const auto& c : cand)
    if (c.second * 100 <= best_cost * 103 && c.first.nch < pick.nch) pick = c.first;
  return pick;
}

}  // namespace wlr

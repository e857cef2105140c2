// Prints the row chunking chosen by wlr_plan.h for the (m, tiles, slots) triples read from
// stdin, one "m tiles slots nch rows" line each (host logic only; no GPU).
#include <cstdio>

#include "wlr_plan.h"

int main() {
  int m, tiles, slots;
  while (std::scanf("%d %d %d", &m, &tiles, &slots) == 3) {
    const wlr::Chunk w = wlr::chunking_waves(m, tiles, slots);
    const wlr::Chunk c = wlr::chunking(m, (size_t)tiles, slots);
    std::printf("%d %d %d %d %d %d %d\n", m, tiles, slots, w.nch, w.rows, c.nch, c.rows);
  }
  return 0;
}

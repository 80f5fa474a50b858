// Host harness of the launch-table dealing rule (paper_2510_27517_gb300/csrc/deal.h),
// built with g++ by tests/test_deal_host.py: the table the engine's host side
// writes for items of the given weights over `grid` blocks.
#include <stdint.h>

#include <vector>

#include "deal.h"

extern "C" int64_t deal_table(const double* weight, int64_t items, int grid, int32_t* table) {
  if (items < 0 || grid < 1) return -1;
  const std::vector<double> w(weight, weight + items);
  const std::vector<int64_t> ord = spai::deal_order(w);
  const int64_t npos = spai::deal_positions(items, grid);
  for (int64_t p = 0; p < npos; ++p) table[p] = -1;
  for (int64_t j = 0; j < items; ++j) table[spai::snake_pos(j, grid)] = (int32_t)ord[j];
  return npos;
}

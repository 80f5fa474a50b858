// Dealing the work items of a launch to the blocks of the persistent engine
// kernel.  Block b of a grid of G blocks runs the launch-table positions
// b, b + G, b + 2G, ...  Items are ranked by decreasing size (stable: equal
// sizes keep their order) and the item of rank j goes to position
// snake_pos(j, G): round r = j / G runs blocks 0 .. G - 1 when r is even and
// G - 1 .. 0 when it is odd, so that members of very different sizes load
// every block about equally.  The last round may be short; its positions that
// no item reaches are holes.  Which block runs an item never changes its
// arithmetic: the kernel's reductions are indexed by the item, not the block.
//
// Plain C++ (host and device), so that a test can build it without CUDA.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <vector>

#if defined(__CUDACC__)
#define SPAI_DEAL_HD __host__ __device__ __forceinline__
#else
#define SPAI_DEAL_HD inline
#endif

namespace spai {

// Table position of the item of rank j.
SPAI_DEAL_HD int64_t snake_pos(int64_t j, int grid) {
  const int64_t r = j / grid, c = j % grid;
  return r * grid + ((r & 1) ? grid - 1 - c : c);
}

// Positions a table of `items` items over `grid` blocks holds (whole rounds).
SPAI_DEAL_HD int64_t deal_positions(int64_t items, int grid) { return (items + grid - 1) / grid * grid; }

// Item indices in dealing order: decreasing weight, stable.
inline std::vector<int64_t> deal_order(const std::vector<double>& weight) {
  std::vector<int64_t> ord(weight.size());
  for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int64_t)i;
  std::stable_sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) { return weight[x] > weight[y]; });
  return ord;
}

}  // namespace spai

// Kernel table entries for the mixed-radix probe sides 96 (24 x 4) and
// 192 (24 x 8).
#include "kernel_sets.cuh"

namespace ptycho {
std::vector<KernelSet> kernel_sets_mixed() {
  return {make_set_noepie<96, 1, 1>(),  make_set_noepie<96, 1, 2>(),  make_set_noepie<96, 1, 4>(),
          make_set_noepie<192, 1, 2>(), make_set_noepie<192, 1, 4>(), make_set_noepie<192, 1, 8>()};
}
}  // namespace ptycho

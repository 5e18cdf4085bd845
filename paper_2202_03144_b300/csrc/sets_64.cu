// Kernel table entries for probe side 64.
#include "kernel_sets.cuh"

namespace ptycho {
std::vector<KernelSet> kernel_sets_64() {
  return {make_set<64, 1, 1>(), make_set<64, 1, 2>(), make_set<64, 1, 4>(), make_set<64, 3, 2>(),
          make_set<64, 3, 4>()};
}
}  // namespace ptycho

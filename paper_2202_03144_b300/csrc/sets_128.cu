// Kernel table entries for probe side 128.
#include "kernel_sets.cuh"

namespace ptycho {
std::vector<KernelSet> kernel_sets_128() {
  return {make_set<128, 1, 2>(), make_set<128, 1, 4>(), make_set<128, 1, 8>(), make_set<128, 3, 4>(),
          make_set<128, 3, 8>()};
}
}  // namespace ptycho

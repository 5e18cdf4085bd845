// Kernel table entries for probe sides 16 and 32.
#include "kernel_sets.cuh"

namespace ptycho {
std::vector<KernelSet> kernel_sets_16_32() {
  return {make_set<16, 1, 1>(), make_set<16, 1, 2>(), make_set<16, 2, 1>(), make_set<16, 3, 1>(),
          make_set<16, 3, 2>(), make_set<32, 1, 1>(), make_set<32, 1, 2>(), make_set<32, 1, 4>(),
          make_set<32, 2, 2>(), make_set<32, 3, 1>(), make_set<32, 3, 4>()};
}
}  // namespace ptycho

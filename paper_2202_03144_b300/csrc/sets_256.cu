// Kernel table entries for probe side 256.
#include "kernel_sets.cuh"

namespace ptycho {
std::vector<KernelSet> kernel_sets_256() {
  return {make_set<256, 1, 4>(), make_set<256, 1, 8>(), make_set<256, 1, 16>()};
}
}  // namespace ptycho

// Kernel table entries for probe side 128.
#include "kernel_sets.cuh"

namespace ptycho {
std::vector<KernelSet> kernel_sets_128() {
  // (128, 3, 16) serves ePIE (a 16-CTA cluster walks the positions 12% faster
  // than 8 CTAs); DM and LSQML run 6% faster at 8, so 16 is no default there
  KernelSet s16 = make_set<128, 3, 16>();
  s16.default_ok = false;
  return {make_set<128, 1, 2>(), make_set<128, 1, 4>(), make_set<128, 1, 8>(), make_set<128, 3, 4>(),
          make_set<128, 3, 8>(), s16};
}
}  // namespace ptycho

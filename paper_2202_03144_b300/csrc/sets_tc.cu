// Kernel table of the tensor-core DFT Fourier pass (64 x 64 detector, one
// probe mode): one kernel per (mode, amplitude format).
#include "dft_tc.cuh"

namespace ptycho {

using TcFourierFn = void (*)(Fourier2Args, const unsigned char*, int);

// The split real-form DFT matrix in the shared-memory byte layout: hi term
// (TC64_AMAT bytes), then lo term.  Entries from sincospi in FP64.
__global__ void k_dft64_matrix(unsigned char* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 128 * 128) return;
  const int m = i / 128, k = i % 128;
  const int f = m & 63, r = k & 63;
  double s, c;
  sincospi((double)((f * r) & 63) / 32.0, &s, &c);  // angle 2 pi f r / 64, reduced
  const double v = (m < 64) ? (k < 64 ? c : s) : (k < 64 ? -s : c);
  const __nv_bfloat16 hi = __float2bfloat16_rn((float)v);
  const __nv_bfloat16 lo = __float2bfloat16_rn((float)(v - (double)__bfloat162float(hi)));
  *reinterpret_cast<__nv_bfloat16*>(out + tc64_off(m, k)) = hi;
  *reinterpret_cast<__nv_bfloat16*>(out + TC64_AMAT + tc64_off(m, k)) = lo;
}


template <int MODE>
TcFourierFn tc64_for_format(int istore) {
  switch (istore) {
    case 0: return k_fourier_tc64<MODE, 0>;
    case 1: return k_fourier_tc64<MODE, 1>;
    case 2: return k_fourier_tc64<MODE, 2>;
    default: return nullptr;
  }
}

// The kernel for a Fourier mode and amplitude format, or NULL.
TcFourierFn tc64_fourier(int mode, int istore) {
  switch (mode) {
    case FM_DM: return tc64_for_format<FM_DM>(istore);
    case FM_CHI: return tc64_for_format<FM_CHI>(istore);
    case FM_CHIP: return tc64_for_format<FM_CHIP>(istore);
    case FM_ERR: return tc64_for_format<FM_ERR>(istore);
    case FM_SIM: return tc64_for_format<FM_SIM>(istore);
    default: return nullptr;
  }
}

// Build the split DFT matrix (2 x 32 KB) into out on the stream.
void tc64_build_matrix(unsigned char* out, cudaStream_t st) {
  k_dft64_matrix<<<(128 * 128 + 255) / 256, 256, 0, st>>>(out);
}

}  // namespace ptycho

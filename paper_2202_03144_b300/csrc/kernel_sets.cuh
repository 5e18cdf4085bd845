// Dispatch table of the per-shape kernels: one entry per compiled
// (M, K, C) = (probe side, probe modes, CTAs per position).
//
// Each entry carries the generic Fourier kernel (mode and amplitude format
// read from the arguments), the ePIE kernel where one exists, and Fourier
// kernels compiled for one mode (DM pass or LSQML residual pass) and one
// amplitude format: with both fixed at compile time the projection loop has
// no per-pixel branches (~9% fewer cycles for the 256^2 residual pass).
//
// The entries are instantiated in several translation units (sets_*.cu),
// compiled in parallel; ptycho_api.cu joins their lists.
#pragma once
#include <vector>

#include "epie.cuh"
#include "epie2.cuh"
#include "fourier2.cuh"
#include "fourier3.cuh"

// 1: the mode-specialised kernels of cluster shapes (C > 1) use the
// asynchronous-transpose form k_fourier3 where its two buffers fit in shared
// memory; 0: k_fourier2 throughout.
#ifndef PT_F3
#define PT_F3 1
#endif

namespace ptycho {

using FourierFn = void (*)(Fourier2Args);

struct KernelSet {
  int M, K, C;
  int NT2, NT_epie;
  size_t smem_fourier, smem_epie;
  FourierFn fourier;       // any mode, any amplitude format
  void (*epie)(EpieArgs);  // null: no ePIE kernel for this shape
  FourierFn spec[5][3];    // [spec_row(mode)][f32, f16, bf16]
  size_t smem_spec;        // dynamic shared memory of the spec kernels: the largest row
  bool default_ok = true;  // a candidate for the default cluster size of DM/LSQML
  void (*epie2)(Epie2Args) = nullptr;  // register-resident ePIE sweep (C > 1), or null
  size_t smem_epie2 = 0;
  size_t smem_row[5] = {};  // dynamic shared memory of each row of spec
};

// Row of KernelSet::spec for a Fourier mode: DM, LSQML residual (amplitude),
// LSQML residual (Poisson), Fourier error, forward model; -1 for modes only
// the generic kernel runs.
__host__ __device__ constexpr int spec_row(int mode) {
  return mode == FM_DM ? 0 : mode == FM_CHI ? 1 : mode == FM_CHIP ? 2 : mode == FM_ERR ? 3 : mode == FM_SIM ? 4 : -1;
}

template <int M, int K, int C, int MODE>
void fill_spec_row(KernelSet& s) {
  constexpr int r = spec_row(MODE);
  if constexpr (C > 1 && PT_F3 && fourier3_smem<F2<M, K, C>, MODE>() <= 227 * 1024) {
    s.spec[r][0] = k_fourier3<M, K, C, MODE, 0>;
    s.spec[r][1] = k_fourier3<M, K, C, MODE, 1>;
    s.spec[r][2] = k_fourier3<M, K, C, MODE, 2>;
    s.smem_row[r] = fourier3_smem<F2<M, K, C>, MODE>();
  } else {
    s.spec[r][0] = k_fourier2<M, K, C, MODE, 0>;
    s.spec[r][1] = k_fourier2<M, K, C, MODE, 1>;
    s.spec[r][2] = k_fourier2<M, K, C, MODE, 2>;
    s.smem_row[r] = fourier2_smem<F2<M, K, C>>();
  }
  if (s.smem_row[r] > s.smem_spec) s.smem_spec = s.smem_row[r];
}

template <int M, int K, int C>
void fill_spec(KernelSet& s) {
  fill_spec_row<M, K, C, FM_DM>(s);
  fill_spec_row<M, K, C, FM_CHI>(s);
  fill_spec_row<M, K, C, FM_CHIP>(s);
  fill_spec_row<M, K, C, FM_ERR>(s);
  fill_spec_row<M, K, C, FM_SIM>(s);
}

template <int M, int K, int C>
KernelSet make_set() {
  using F = FCfg<M, K, C>;
  using G = F2<M, K, C>;
  KernelSet s{M, K, C, G::NT, F::NT, fourier2_smem<G>(), epie_smem<F>(), k_fourier2<M, K, C>, k_epie<M, K, C>, {}, 0, true};
  fill_spec<M, K, C>(s);
  if constexpr (C > 1 && epie2_smem<G>() <= 227 * 1024) {
    s.epie2 = k_epie2<M, K, C>;
    s.smem_epie2 = epie2_smem<G>();
  }
  return s;
}

// mixed-radix sizes: DM / LSQML / error / forward model only (no ePIE kernel)
template <int M, int K, int C>
KernelSet make_set_noepie() {
  using G = F2<M, K, C>;
  KernelSet s{M, K, C, G::NT, 0, fourier2_smem<G>(), 0, k_fourier2<M, K, C>, nullptr, {}, 0, true};
  fill_spec<M, K, C>(s);
  return s;
}

std::vector<KernelSet> kernel_sets_16_32();  // M = 16, 32
std::vector<KernelSet> kernel_sets_64();
std::vector<KernelSet> kernel_sets_128();
std::vector<KernelSet> kernel_sets_256();
std::vector<KernelSet> kernel_sets_mixed();  // M = 96, 192

}  // namespace ptycho

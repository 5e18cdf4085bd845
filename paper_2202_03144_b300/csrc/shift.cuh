// Sub-pixel probe shifts (Fourier shift theorem).
//
// Positions quantised to 1/S pixel (S even) are an integer corner plus a
// shift delta = (b - S/2) / S per axis, b in [0, S).  The probe seen at such
// a position is T_delta P with
//     F(T_delta P)(f) = F(P)(f) exp(-2 pi i (f_y dy + f_x dx)),
// f = k/M for k < M/2 and (k - M)/M otherwise, so (T P)(u) = P(u - delta) for
// a band-limited probe.  T is separable: a shift of every row along x, then of
// every column along y, each a length-M FFT, a phase ramp and an inverse FFT.
//
// Two operations, each two launches over lines held in shared memory:
//   build: tab[by S + bx][k] = T_(dy(by), dx(bx)) src[k]        (fan out)
//          rows: tmp[bx][k] = T_x(dx(bx)) src[k];  cols: tab from tmp
//   sum:   out[k] = sum_b T_-delta(b) bins[b][k]                 (fan in, the
//          adjoint of build summed over the bins, in fixed order)
//          cols: tmp[bx][k] = sum_by T_y(-dy(by)) bins[by S + bx][k]
//          rows: out[k]     = sum_bx T_x(-dx(bx)) tmp[bx][k]
// The fan-in sums are taken in the frequency domain (one inverse FFT per line)
// and skip bins that hold no position.
//
// Single-shift form (one != 0, the sub-pixel ePIE sweep): the build kernels
// shift the K source arrays by one delta = (bye - S/2, bxe - S/2) / S into
// slot 0, bye and bxe any integers (a bin, a reflected bin for the adjoint, or
// the difference of two bins), and the column pass may add its result to the
// output instead of storing it.
#pragma once
#include "common.cuh"
#include "fourier2.cuh"

namespace ptycho {

constexpr int SH_NT = 128;

template <int M, int LN>
struct ShCfg {
  static constexpr int R1 = radix1(M), R2 = M / R1;
  static constexpr int PITCH = M + 1;           // line pitch in shared memory (float2)
  static constexpr int E = LN * M / SH_NT;      // elements per thread
  static_assert(R1 * R2 == M, "radix split");
  static_assert((LN * M) % SH_NT == 0 && E >= 1, "lines x length must split over the threads");
};

// In-place length-M FFT of LN lines at s[l * PITCH + i] (unnormalised both ways).
template <int M, int LN, bool INV>
__device__ __forceinline__ void sh_fft(float2* s, const float2* tw) {
  using C = ShCfg<M, LN>;
  stockham_pass<M, C::R1, 1, LN, LN, 0, C::PITCH, 1, SH_NT, INV>(s, tw);
  if constexpr (C::R2 > 1) stockham_pass<M, C::R2, C::R1, LN, LN, 0, C::PITCH, 1, SH_NT, INV>(s, tw);
}

// exp(-2 pi i f delta) / M with f the signed frequency of bin k and
// delta = sgn (b - S/2) / S:  the argument is -2 kk (b - S/2) sgn / (M S) half-turns.
__device__ __forceinline__ float2 sh_phase(int k, int M, int b, int S, int sgn) {
  const int kk = k < M / 2 ? k : k - M;
  const int n = kk * (2 * b - S) * sgn;
  float sn, cs;
  sincospif(-(float)n / (float)(M * S), &sn, &cs);
  const float inv = 1.f / (float)M;
  return make_float2(cs * inv, sn * inv);
}

template <int M>
__device__ __forceinline__ void sh_load_tw(float2* tw_s, const float2* tw) {
  for (int i = threadIdx.x; i < M; i += SH_NT) tw_s[i] = tw[i];
}

// build, rows: grid (K*M/LN, S) (single shift: (K*M/LN, 1)).
// tmp[bx][k][y][:] = T_x(dx(bx)) src[k][y][:]
template <int M, int LN>
__global__ void __launch_bounds__(SH_NT) k_shift_build_rows(const float2* __restrict__ src, float2* __restrict__ tmp,
                                                            int K, int S, const float2* __restrict__ tw, int one,
                                                            int bxe) {
  using C = ShCfg<M, LN>;
  __shared__ float2 s[LN * C::PITCH];
  __shared__ float2 tw_s[M];
  sh_load_tw<M>(tw_s, tw);
  pdl_wait();
  pdl_launch();
  const int row0 = blockIdx.x * LN;
  const int bx = one ? bxe : (int)blockIdx.y;
  const int slot = one ? 0 : bx;
  for (int e = threadIdx.x; e < LN * M; e += SH_NT) {
    const int l = e / M, i = e % M;
    s[l * C::PITCH + i] = src[(size_t)(row0 + l) * M + i];
  }
  __syncthreads();
  sh_fft<M, LN, false>(s, tw_s);
  for (int e = threadIdx.x; e < LN * M; e += SH_NT) {
    const int l = e / M, i = e % M;
    s[l * C::PITCH + i] = cmul(s[l * C::PITCH + i], sh_phase(i, M, bx, S, 1));
  }
  __syncthreads();
  sh_fft<M, LN, true>(s, tw_s);
  float2* dst = tmp + (size_t)slot * K * M * M;
  for (int e = threadIdx.x; e < LN * M; e += SH_NT) {
    const int l = e / M, i = e % M;
    dst[(size_t)(row0 + l) * M + i] = s[l * C::PITCH + i];
  }
}

// build, columns: grid (M/LN, K, S*S) (single shift: (M/LN, K, 1)).
// tab[by S + bx][k][:][x] = T_y(dy(by)) tmp[bx][k][:][x]  (accumulate: +=),
// times bscale[b][pixel] when bscale is given (the DM probe solve's per-bin
// |O|^2 sums)
template <int M, int LN>
__global__ void __launch_bounds__(SH_NT) k_shift_build_cols(const float2* __restrict__ tmp, float2* __restrict__ tab,
                                                            int K, int S, const float2* __restrict__ tw, int one,
                                                            int bye, int accumulate,
                                                            const float* __restrict__ bscale) {
  using C = ShCfg<M, LN>;
  __shared__ float2 s[LN * C::PITCH];
  __shared__ float2 tw_s[M];
  sh_load_tw<M>(tw_s, tw);
  pdl_wait();
  pdl_launch();
  const int c0 = blockIdx.x * LN, k = blockIdx.y;
  const int b = one ? 0 : (int)blockIdx.z;
  const int by = one ? bye : b / S, bx = b % S;
  const int in_slot = one ? 0 : bx, out_slot = one ? 0 : b;
  const float2* in = tmp + ((size_t)in_slot * K + k) * M * M;
  for (int e = threadIdx.x; e < LN * M; e += SH_NT) {
    const int i = e / LN, l = e % LN;   // row i, column c0 + l
    s[l * C::PITCH + i] = in[(size_t)i * M + c0 + l];
  }
  __syncthreads();
  sh_fft<M, LN, false>(s, tw_s);
  for (int e = threadIdx.x; e < LN * M; e += SH_NT) {
    const int l = e / M, i = e % M;
    s[l * C::PITCH + i] = cmul(s[l * C::PITCH + i], sh_phase(i, M, by, S, 1));
  }
  __syncthreads();
  sh_fft<M, LN, true>(s, tw_s);
  float2* out = tab + ((size_t)out_slot * K + k) * M * M;
  const float* sc = bscale ? bscale + (size_t)b * M * M : nullptr;
  for (int e = threadIdx.x; e < LN * M; e += SH_NT) {
    const int i = e / LN, l = e % LN;
    const size_t o = (size_t)i * M + c0 + l;
    float2 v = s[l * C::PITCH + i];
    if (sc) v = cscale(v, sc[o]);
    out[o] = accumulate ? cadd(out[o], v) : v;
  }
}

// Single shift, columns, all K modes of LN columns per CTA (the sub-pixel
// ePIE frame change): grid (M/LN).  dst[k][:][x] = T_y(dy(bye)) tmp[k][:][x]
// for the CTA's columns x, and mx[blockIdx.x] = (max sum_k |dst_k|^2,
// max |O_j|^2) over those columns: the partial probe and object maxima of the
// ePIE step at position j (patch corner pos[j]).
template <int M, int LN, int K>
__global__ void __launch_bounds__(SH_NT) k_shift_one_cols(const float2* __restrict__ tmp, float2* __restrict__ dst,
                                                          int S, const float2* __restrict__ tw, int bye,
                                                          const float2* __restrict__ O, int nx,
                                                          const int2* __restrict__ pos, int j,
                                                          float2* __restrict__ mx) {
  constexpr int L = K * LN;   // line l = k LN + (column - c0)
  using C = ShCfg<M, L>;
  __shared__ float2 s[L * C::PITCH];
  __shared__ float2 tw_s[M];
  __shared__ float red[32];
  sh_load_tw<M>(tw_s, tw);
  pdl_wait();
  pdl_launch();
  const int c0 = blockIdx.x * LN;
  for (int e = threadIdx.x; e < L * M; e += SH_NT) {
    const int i = e / L, l = e % L;
    s[l * C::PITCH + i] = tmp[((size_t)(l / LN) * M + i) * M + c0 + l % LN];
  }
  const int2 p = pos[j];
  float om = 0.f;
  for (int e = threadIdx.x; e < LN * M; e += SH_NT)
    om = fmaxf(om, cabs2(O[(size_t)(p.x + e / LN) * nx + p.y + c0 + e % LN]));
  __syncthreads();
  sh_fft<M, L, false>(s, tw_s);
  for (int e = threadIdx.x; e < L * M; e += SH_NT) {
    const int l = e / M, i = e % M;
    s[l * C::PITCH + i] = cmul(s[l * C::PITCH + i], sh_phase(i, M, bye, S, 1));
  }
  __syncthreads();
  sh_fft<M, L, true>(s, tw_s);
  float pm = 0.f;
  for (int e = threadIdx.x; e < LN * M; e += SH_NT) {
    const int i = e / LN, lc = e % LN;
    float a = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float2 v = s[(k * LN + lc) * C::PITCH + i];
      dst[((size_t)k * M + i) * M + c0 + lc] = v;
      a += cabs2(v);
    }
    pm = fmaxf(pm, a);
  }
  pm = block_max_f<SH_NT>(pm, red);
  om = block_max_f<SH_NT>(om, red);
  if (threadIdx.x == 0) mx[blockIdx.x] = make_float2(pm, om);
}

// sum, columns: grid (M/LN, K, S).  tmp[bx][k][:][x] = sum_by T_y(-dy(by)) bins[by S + bx][k][:][x];
// bgrp[b] == bgrp[b + 1] marks a bin without positions (its sum is zero).
template <int M, int LN>
__global__ void __launch_bounds__(SH_NT) k_shift_sum_cols(const float2* __restrict__ bins, float2* __restrict__ tmp,
                                                          int K, int S, const int* __restrict__ bgrp,
                                                          const float2* __restrict__ tw) {
  using C = ShCfg<M, LN>;
  __shared__ float2 s[LN * C::PITCH];
  __shared__ float2 tw_s[M];
  sh_load_tw<M>(tw_s, tw);
  const int c0 = blockIdx.x * LN, k = blockIdx.y, bx = blockIdx.z;
  float2 acc[C::E];
#pragma unroll
  for (int q = 0; q < C::E; ++q) acc[q] = make_float2(0.f, 0.f);
  for (int by = 0; by < S; ++by) {
    const int b = by * S + bx;
    if (bgrp[b] == bgrp[b + 1]) continue;   // uniform over the CTA
    const float2* in = bins + ((size_t)b * K + k) * M * M;
    __syncthreads();
    for (int e = threadIdx.x; e < LN * M; e += SH_NT) {
      const int i = e / LN, l = e % LN;
      s[l * C::PITCH + i] = in[(size_t)i * M + c0 + l];
    }
    __syncthreads();
    sh_fft<M, LN, false>(s, tw_s);
#pragma unroll
    for (int q = 0; q < C::E; ++q) {
      const int e = threadIdx.x + q * SH_NT;
      const int l = e / M, i = e % M;
      const float2 t = cmul(s[l * C::PITCH + i], sh_phase(i, M, by, S, -1));
      acc[q] = cadd(acc[q], t);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < C::E; ++q) {
    const int e = threadIdx.x + q * SH_NT;
    s[(e / M) * C::PITCH + e % M] = acc[q];
  }
  __syncthreads();
  sh_fft<M, LN, true>(s, tw_s);
  float2* out = tmp + ((size_t)bx * K + k) * M * M;
  for (int e = threadIdx.x; e < LN * M; e += SH_NT) {
    const int i = e / LN, l = e % LN;
    out[(size_t)i * M + c0 + l] = s[l * C::PITCH + i];
  }
}

// sum, rows: grid (K*M/LN).  out[k][y][:] = sum_bx T_x(-dx(bx)) tmp[bx][k][y][:]
template <int M, int LN>
__global__ void __launch_bounds__(SH_NT) k_shift_sum_rows(const float2* __restrict__ tmp, float2* __restrict__ out,
                                                          int K, int S, const float2* __restrict__ tw) {
  using C = ShCfg<M, LN>;
  __shared__ float2 s[LN * C::PITCH];
  __shared__ float2 tw_s[M];
  sh_load_tw<M>(tw_s, tw);
  const int row0 = blockIdx.x * LN;
  float2 acc[C::E];
#pragma unroll
  for (int q = 0; q < C::E; ++q) acc[q] = make_float2(0.f, 0.f);
  for (int bx = 0; bx < S; ++bx) {
    const float2* in = tmp + (size_t)bx * K * M * M;
    __syncthreads();
    for (int e = threadIdx.x; e < LN * M; e += SH_NT) {
      const int l = e / M, i = e % M;
      s[l * C::PITCH + i] = in[(size_t)(row0 + l) * M + i];
    }
    __syncthreads();
    sh_fft<M, LN, false>(s, tw_s);
#pragma unroll
    for (int q = 0; q < C::E; ++q) {
      const int e = threadIdx.x + q * SH_NT;
      const int l = e / M, i = e % M;
      acc[q] = cadd(acc[q], cmul(s[l * C::PITCH + i], sh_phase(i, M, bx, S, -1)));
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < C::E; ++q) {
    const int e = threadIdx.x + q * SH_NT;
    s[(e / M) * C::PITCH + e % M] = acc[q];
  }
  __syncthreads();
  sh_fft<M, LN, true>(s, tw_s);
  for (int e = threadIdx.x; e < LN * M; e += SH_NT) {
    const int l = e / M, i = e % M;
    out[(size_t)(row0 + l) * M + i] = s[l * C::PITCH + i];
  }
}

}  // namespace ptycho

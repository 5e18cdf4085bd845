// Shared-memory Fourier building blocks of the single-CTA ePIE kernel
// (k_epie): the per-shape configuration FCfg, Stockham passes over lines held
// in shared memory, the cluster transposes between the column-distributed and
// the row-distributed layouts, and the modulus projection in place.
//
// Work split.  The K x M x M complex exit waves of one position are shared by
// the C CTAs of a cluster (C = 1, 2, 4, 8).  Two shared-memory layouts:
//   layout A (column-distributed): CTA c holds columns [c W, (c+1) W),
//            all M rows, all K modes:  A[k][row][colL], pitch PA;
//   layout B (row-distributed):    CTA c holds rows [c H, (c+1) H), all M
//            columns, all K modes:    B[k][rowL][col],  pitch PB = M + 1.
// W = H = M / C.  The forward transform does column FFTs in layout A,
// transposes A -> B through distributed shared memory (each element crosses
// the cluster once), then row FFTs in layout B.  The projection needs all K
// modes of a Fourier pixel, which layout B holds locally.  The inverse runs
// the same way backwards (rows in B, transpose B -> A, columns in A).
//
// The projection writes the Fourier difference D = Pi(Z) - Z (scaled by
// 1/M^2) instead of Pi(Z), so that by linearity
//   chi = F^-1 Pi(F phi) - phi = F^-1 D.
#pragma once
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"

namespace ptycho {
namespace cg = cooperative_groups;

// DM pass, LSQML residual (amplitude likelihood), Fourier error, forward
// model, LSQML residual with the Poisson-likelihood correction.
enum FourierMode : int { FM_DM = 0, FM_CHI = 1, FM_ERR = 2, FM_SIM = 3, FM_CHIP = 4 };

__host__ __device__ constexpr int choose_E(int L) {
  // elements per thread: a power of two <= 16 giving a whole number of warps
  for (int E = 16; E >= 2; E >>= 1)
    if (L % E == 0 && (L / E) % 32 == 0 && L / E <= 1024) return E;
  return 16;
}

template <int M_, int K_, int C_>
struct FCfg {
  static constexpr int M = M_, K = K_, C = C_;
  static constexpr int W = M / C, H = M / C;
  static constexpr int L = K * M * M / C;
  static constexpr int E = choose_E(L);
  static constexpr int NT = L / E;
  static constexpr int PA = (C == 1) ? M + 1 : W;
  static constexpr int PB = M + 1;
  static constexpr int SA = K * M * PA, SB = K * H * PB;
  static constexpr int SBUF = SA > SB ? SA : SB;
  static constexpr int NRED = 64;  // doubles of reduction scratch
  static_assert(M % C == 0, "M divisible by C");
  static_assert(NT % 32 == 0 && NT <= 1024, "thread count");
  static_assert(L % E == 0, "elements per thread");
};

// Shared memory (bytes) of the Fourier kernel: data + twiddles + reduction.
template <class F>
__host__ __device__ constexpr size_t fourier_smem() {
  return (size_t)(F::SBUF + F::M) * sizeof(float2) + F::NRED * sizeof(double);
}

struct FourierArgs {
  const float2* O;        // object [ny][nx]
  int nx;
  const float2* P;        // probe [K][M][M]
  const int2* pos;        // [J] (y, x) integer top-left corners
  float2* X;              // DM: psi (in/out); CHI: chi (out)   [J][K][M][M]
  const void* amp;        // stored sqrt(I) in FFT order [J][M][M]
  const float* amp_scale; // per-frame scale (16-bit storage)
  int istore;             // 0 f32, 1 f16, 2 bf16
  float* I_out;           // SIM: detector-centred intensities [J][M][M]
  double2* err_part;      // ERR: per-CTA (sum (A - a)^2, sum a^2), [J*C]
  const float2* tw;       // exp(-2 pi i n / M), n < M
  int j0;                 // first position of this launch
  int mode;
};

__device__ __forceinline__ float load_amp(const FourierArgs& a, size_t idx, int j) {
  if (a.istore == 0) return __ldg(reinterpret_cast<const float*>(a.amp) + idx);
  float q;
  if (a.istore == 1) q = __half2float(reinterpret_cast<const __half*>(a.amp)[idx]);
  else q = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(a.amp)[idx]);
  return q * __ldg(a.amp_scale + j);
}

// Layout A -> layout B through distributed shared memory.  Every CTA first
// waits until all CTAs finished writing layout A (SYNC_BEFORE), pulls its
// rows from the owners of each column block into registers, waits until
// every CTA finished reading, then overwrites its own buffer.
template <class F, bool SYNC_BEFORE>
__device__ __forceinline__ void transpose_A_to_B(float2* buf, int c) {
  cg::cluster_group cl = cg::this_cluster();
  float2 v[F::E];
  if (SYNC_BEFORE) cl.sync();
#pragma unroll
  for (int q = 0; q < F::E; ++q) {
    const int e = threadIdx.x + q * F::NT;
    const int col = e % F::M, rowL = (e / F::M) % F::H, k = e / (F::M * F::H);
    const float2* rb = cl.map_shared_rank(buf, col / F::W);
    v[q] = rb[k * F::M * F::PA + (c * F::H + rowL) * F::PA + (col % F::W)];
  }
  cl.sync();
#pragma unroll
  for (int q = 0; q < F::E; ++q) {
    const int e = threadIdx.x + q * F::NT;
    const int col = e % F::M, rowL = (e / F::M) % F::H, k = e / (F::M * F::H);
    buf[k * F::H * F::PB + rowL * F::PB + col] = v[q];
  }
  __syncthreads();
}

template <class F>
__device__ __forceinline__ void transpose_B_to_A(float2* buf, int c) {
  cg::cluster_group cl = cg::this_cluster();
  float2 v[F::E];
  cl.sync();
#pragma unroll
  for (int q = 0; q < F::E; ++q) {
    const int e = threadIdx.x + q * F::NT;
    const int colL = e % F::W, row = (e / F::W) % F::M, k = e / (F::W * F::M);
    const float2* rb = cl.map_shared_rank(buf, row / F::H);
    v[q] = rb[k * F::H * F::PB + (row % F::H) * F::PB + c * F::W + colL];
  }
  cl.sync();
#pragma unroll
  for (int q = 0; q < F::E; ++q) {
    const int e = threadIdx.x + q * F::NT;
    const int colL = e % F::W, row = (e / F::W) % F::M, k = e / (F::W * F::M);
    buf[k * F::M * F::PA + row * F::PA + colL] = v[q];
  }
  __syncthreads();
}

// Forward 2-D FFT of the cluster's tile: columns in layout A, then rows in B.
template <class F, bool SYNC_BEFORE = true>
__device__ __forceinline__ void fft2_forward(float2* buf, const float2* tw, int c) {
  fft_lines<F::M, F::E, F::K * F::W, F::W, F::M * F::PA, 1, F::PA, F::NT, false>(buf, tw);
  if constexpr (F::C > 1) transpose_A_to_B<F, SYNC_BEFORE>(buf, c);
  fft_lines<F::M, F::E, F::K * F::H, F::K * F::H, 0, F::PB, 1, F::NT, false>(buf, tw);
}

// Inverse (unnormalised) 2-D FFT: rows in layout B, then columns in A.
template <class F>
__device__ __forceinline__ void fft2_inverse(float2* buf, const float2* tw, int c) {
  fft_lines<F::M, F::E, F::K * F::H, F::K * F::H, 0, F::PB, 1, F::NT, true>(buf, tw);
  if constexpr (F::C > 1) transpose_B_to_A<F>(buf, c);
  fft_lines<F::M, F::E, F::K * F::W, F::W, F::M * F::PA, 1, F::PA, F::NT, true>(buf, tw);
}

// Modulus projection in layout B, writing D = (Pi(Z) - Z) / M^2 in place.
// A = sqrt(sum_k |Z_k|^2); masked (a < 0): D = 0; A <= 1e-20: D = -Z.
template <class F>
__device__ __forceinline__ void project_difference(float2* buf, const FourierArgs& a, int j, int c) {
  constexpr float inv = 1.0f / (float)(F::M * F::M);
  for (int px = threadIdx.x; px < F::H * F::M; px += F::NT) {
    const int rowL = px / F::M, col = px % F::M;
    const int ky = c * F::H + rowL;
    float2 z[F::K];
    float A2 = 0.f;
#pragma unroll
    for (int k = 0; k < F::K; ++k) {
      z[k] = buf[k * F::H * F::PB + rowL * F::PB + col];
      A2 += cabs2(z[k]);
    }
    const float amp = load_amp(a, ((size_t)j * F::M + ky) * F::M + col, j);
    float f = 0.f;
    if (amp >= 0.f) {
      const float A = sqrtf(A2);
      f = ((A > 1e-20f) ? amp / A : 0.f) - 1.f;
    }
    f *= inv;
#pragma unroll
    for (int k = 0; k < F::K; ++k) buf[k * F::H * F::PB + rowL * F::PB + col] = cscale(z[k], f);
  }
  __syncthreads();
}

}  // namespace ptycho

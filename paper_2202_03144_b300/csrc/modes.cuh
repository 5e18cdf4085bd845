// Probe-mode orthogonalisation (Thibault & Menzel 2013, cited in Sec. 1):
// rotate the K probe modes into the eigenbasis of their Gram matrix
//   G[l][k] = <P_l, P_k> = sum_u conj(P_l(u)) P_k(u)
// so that they are mutually orthogonal with decreasing powers; the DM exit
// waves are mixed with the same unitary.  All on the device, no host sync:
//   k_mode_gram   one CTA per (l, k): FP64 block sum over the M^2 pixels
//   k_mode_eig    one thread: cyclic Jacobi on the real 2K x 2K symmetric
//                 form [[Re G, -Im G], [Im G, Re G]] of the Hermitian G (each
//                 eigenvalue appears twice; one vector per pair gives the
//                 complex eigenvector x + i y), decreasing order, the phase
//                 of each eigenvector fixed so that its entry of largest
//                 modulus (the first on a tie) is real positive
//   k_mode_mix    X'_m(u) = sum_l V[l][m] X_l(u) for every frame of X
#pragma once
#include "common.cuh"

namespace ptycho {

constexpr int MODE_KMAX = 3;

__global__ void __launch_bounds__(256) k_mode_gram(const float2* __restrict__ P, int K, int MM, double2* __restrict__ G) {
  __shared__ double red[32];
  const int l = blockIdx.x / K, k = blockIdx.x % K;
  double re = 0.0, im = 0.0;
  for (int u = threadIdx.x; u < MM; u += 256) {
    const float2 a = P[(size_t)l * MM + u], b = P[(size_t)k * MM + u];
    // conj(a) * b
    re += (double)a.x * b.x + (double)a.y * b.y;
    im += (double)a.x * b.y - (double)a.y * b.x;
  }
  re = block_sum_d<256>(re, red);
  im = block_sum_d<256>(im, red);
  if (threadIdx.x == 0) G[l * K + k] = make_double2(re, im);
}

// V[l][m] (complex, FP64) from G (K x K, K <= MODE_KMAX).
__global__ void k_mode_eig(const double2* __restrict__ G, int K, double2* __restrict__ V) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  constexpr int NMAX = 2 * MODE_KMAX;
  const int n = 2 * K;
  double S[NMAX][NMAX], E[NMAX][NMAX];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const int a = i % K, b = j % K;
      const double2 g = G[a * K + b];
      double v;
      if ((i < K) == (j < K)) v = g.x;   // Re G on both diagonal blocks
      else if (i >= K) v = g.y;          // lower-left:  Im G
      else v = -g.y;                     // upper-right: -Im G
      S[i][j] = v;
      E[i][j] = i == j ? 1.0 : 0.0;
    }
  // symmetrise against rounding of G
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) S[i][j] = S[j][i] = 0.5 * (S[i][j] + S[j][i]);
  double scale = 0.0;
  for (int i = 0; i < n; ++i) scale = fmax(scale, fabs(S[i][i]));
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += S[p][q] * S[p][q];
    if (off <= 1e-30 * scale * scale) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        if (S[p][q] == 0.0) continue;
        // rotation zeroing S[p][q] (symmetric Schur decomposition)
        const double theta = (S[q][q] - S[p][p]) / (2.0 * S[p][q]);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        for (int r = 0; r < n; ++r) {
          const double sp = S[r][p], sq = S[r][q];
          S[r][p] = c * sp - s * sq;
          S[r][q] = s * sp + c * sq;
        }
        for (int r = 0; r < n; ++r) {
          const double sp = S[p][r], sq = S[q][r];
          S[p][r] = c * sp - s * sq;
          S[q][r] = s * sp + c * sq;
        }
        for (int r = 0; r < n; ++r) {
          const double ep = E[r][p], eq = E[r][q];
          E[r][p] = c * ep - s * eq;
          E[r][q] = s * ep + c * eq;
        }
      }
  }
  // eigenvalues in decreasing order (stable selection sort of indices)
  int idx[NMAX];
  for (int i = 0; i < n; ++i) idx[i] = i;
  for (int i = 0; i < n; ++i) {
    int b = i;
    for (int j = i + 1; j < n; ++j)
      if (S[idx[j]][idx[j]] > S[idx[b]][idx[b]]) b = j;
    const int t = idx[i];
    idx[i] = idx[b];
    idx[b] = t;
  }
  for (int m = 0; m < K; ++m) {
    const int col = idx[2 * m];  // one vector of each degenerate pair
    double2 v[MODE_KMAX];
    double nrm = 0.0;
    for (int l = 0; l < K; ++l) {
      v[l] = make_double2(E[l][col], E[l + K][col]);
      nrm += v[l].x * v[l].x + v[l].y * v[l].y;
    }
    nrm = sqrt(nrm);
    int imax = 0;
    double amax = -1.0;
    for (int l = 0; l < K; ++l) {
      const double a = sqrt(v[l].x * v[l].x + v[l].y * v[l].y);
      if (a > amax * (1.0 + 1e-12)) {
        amax = a;
        imax = l;
      }
    }
    // multiply by conj(v[imax]) / |v[imax]| and normalise
    const double2 ph = make_double2(v[imax].x / amax, -v[imax].y / amax);
    for (int l = 0; l < K; ++l) {
      const double2 w = make_double2(v[l].x * ph.x - v[l].y * ph.y, v[l].x * ph.y + v[l].y * ph.x);
      V[l * K + m] = make_double2(w.x / nrm, w.y / nrm);
    }
  }
}

// X'_m(u) = sum_l V[l][m] X_l(u) for nf frames of K modes of MM pixels.
__global__ void k_mode_mix(float2* __restrict__ X, size_t nf, int K, int MM, const double2* __restrict__ V) {
  __shared__ float2 v[MODE_KMAX * MODE_KMAX];
  if (threadIdx.x < K * K) v[threadIdx.x] = make_float2((float)V[threadIdx.x].x, (float)V[threadIdx.x].y);
  __syncthreads();
  const size_t n = nf * (size_t)MM;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t f = i / MM, u = i % MM;
    float2* base = X + f * K * MM + u;
    float2 x[MODE_KMAX];
    for (int l = 0; l < K; ++l) x[l] = base[(size_t)l * MM];
    for (int m = 0; m < K; ++m) {
      float2 acc = make_float2(0.f, 0.f);
      for (int l = 0; l < K; ++l) acc = cadd(acc, cmul(v[l * K + m], x[l]));
      base[(size_t)m * MM] = acc;
    }
  }
}

}  // namespace ptycho

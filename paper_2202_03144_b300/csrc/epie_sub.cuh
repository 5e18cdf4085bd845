// Sub-pixel ePIE: the per-position steps around the Fourier pass.  The probe
// is held in the frame of position j, P_j = T_delta_j P, and
// Delta = F^-1 Pi(F(P_j O_j)) - P_j O_j comes from the residual pass:
//   pmax = max_u sum_k |P_j,k(u)|^2,  omax = max_u |O_j(u)|^2      (k_epie_sub_max, or
//        the frame change's column pass when the frame changes: k_shift_one_cols)
//   O_j   += alpha sum_k conj(P_j,k) Delta_k / pmax               (k_epie_sub_update)
//   P_j,k += beta conj(O_j_old) Delta_k / omax                    (k_epie_sub_update)
// -- the probe step in position j's frame; T_-delta_j of it is the step of
// the unshifted probe, and the frame is changed by shifts between positions.
#pragma once
#include "common.cuh"

namespace ptycho {

constexpr int EPS_NT = 256;
constexpr int EPS_MX = 32;   // CTAs of the maxima kernel (partial maxima, reduced by the update)
constexpr int EPS_MX_CAP = 256;  // partial maxima buffer: EPS_MX, or one per column block of the frame change

// grid EPS_MX: out[b] = (max sum_k |P_j,k|^2, max |O_j|^2) over CTA b's pixels
template <int K>
__global__ void __launch_bounds__(EPS_NT) k_epie_sub_max(const float2* __restrict__ Pj, const float2* __restrict__ O,
                                                         int nx, const int2* __restrict__ pos, int j, int M,
                                                         float2* __restrict__ out) {
  __shared__ float red[32];
  pdl_wait();
  pdl_launch();
  const int2 p = pos[j];
  const int MM = M * M;
  float pm = 0.f, om = 0.f;
  for (int u = blockIdx.x * EPS_NT + threadIdx.x; u < MM; u += EPS_MX * EPS_NT) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) s += cabs2(Pj[(size_t)k * MM + u]);
    pm = fmaxf(pm, s);
    om = fmaxf(om, cabs2(O[(size_t)(p.x + u / M) * nx + p.y + u % M]));
  }
  pm = block_max_f<EPS_NT>(pm, red);
  om = block_max_f<EPS_NT>(om, red);
  if (threadIdx.x == 0) out[blockIdx.x] = make_float2(pm, om);
}

// grid MM / 256 (rounded up), one pixel per thread: the pixel's loads are
// issued before the partial maxima are reduced
template <int K>
__global__ void __launch_bounds__(256) k_epie_sub_update(float2* __restrict__ O, int nx, const int2* __restrict__ pos,
                                                         int j, int M, float2* __restrict__ Pj,
                                                         const float2* __restrict__ D, const float2* __restrict__ mx,
                                                         int nmx, float alpha, float beta, int upd) {
  __shared__ float red[32];
  __shared__ float2 tot;
  pdl_wait();
  pdl_launch();
  const int2 p = pos[j];
  const int MM = M * M;
  const int u = blockIdx.x * 256 + threadIdx.x;
  const bool act = u < MM;
  float2* op = nullptr;
  float2 o = make_float2(0.f, 0.f), d[K], pk[K];
  if (act) {
    op = O + (size_t)(p.x + u / M) * nx + p.y + u % M;
    o = *op;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      d[k] = D[(size_t)k * MM + u];
      pk[k] = Pj[(size_t)k * MM + u];
    }
  }
  float pmax = 0.f, omax = 0.f;
  for (int b = threadIdx.x; b < nmx; b += 256) {
    pmax = fmaxf(pmax, mx[b].x);
    omax = fmaxf(omax, mx[b].y);
  }
  pmax = block_max_f<256>(pmax, red);
  omax = block_max_f<256>(omax, red);
  if (threadIdx.x == 0) tot = make_float2(pmax, omax);
  __syncthreads();
  pmax = tot.x;
  omax = tot.y;
  if (!act) return;
  const float sa = pmax > 0.f ? alpha / pmax : 0.f;
  const float sb = (upd && omax > 0.f) ? beta / omax : 0.f;
  float2 num = make_float2(0.f, 0.f);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    num = cadd(num, cconjmul(pk[k], d[k]));
    if (upd) Pj[(size_t)k * MM + u] = cadd(pk[k], cscale(cconjmul(o, d[k]), sb));
  }
  *op = cadd(o, cscale(num, sa));
}

}  // namespace ptycho

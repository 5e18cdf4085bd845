// ePIE (Maiden & Rodenburg 2009, named in the ptychopy paper's Abstract and
// Sec. 1; multi-mode probe as in Thibault & Menzel 2013) as ONE persistent
// thread-block cluster that walks the positions of every iteration in the
// host-given order.  ePIE is sequential by definition -- each position's
// update feeds the next -- so the whole GPU cannot help one position without
// grid-wide syncs; a cluster of C CTAs with hardware cluster barriers gives
// the lowest latency per position instead.
//
// CTA c owns columns [c W, (c+1) W) of the patch and therefore, for the whole
// launch, the same columns of every probe mode: they stay in shared memory
// (exact FP32 values) and are written back once at the end.  The object lives
// in global memory (L2-resident); it is read and written with L2-coherent
// (.cg) accesses, and a cluster barrier with release/acquire semantics
// separates consecutive positions.
//
// Per position j (values from before this position's update):
//   psi_k = P_k O_j;  Delta_k = F^-1 Pi(F psi)_k - psi_k  (fused Fourier step)
//   O_j  += alpha sum_k conj(P_k) Delta_k / max_u sum_k |P_k(u)|^2
//   P_k  += beta conj(O_j) Delta_k / max_u |O_j(u)|^2      (t >= probe_start)
#pragma once
#include "fourier.cuh"

namespace ptycho {

struct EpieArgs {
  float2* O;              // object [ny][nx] (in/out)
  int nx;
  float2* P;              // probe [K][M][M] (in/out)
  const int2* pos;        // [J]
  const void* amp;
  const float* amp_scale;
  int istore;
  const float2* tw;
  const int* order;       // [n_iter][J] visiting order
  int J, n_iter;
  long long t0;           // iteration index of the first iteration
  int probe_start;
  float alpha, beta;
};

template <class F>
__host__ __device__ constexpr size_t epie_smem() {
  return fourier_smem<F>() + (size_t)F::K * F::M * F::W * sizeof(float2) + 8 * sizeof(float);
}

template <int M, int K, int C>
__global__ void __launch_bounds__(FCfg<M, K, C>::NT) k_epie(EpieArgs a) {
  using F = FCfg<M, K, C>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* buf = reinterpret_cast<float2*>(smem_raw);
  float2* tw = buf + F::SBUF;
  double* red = reinterpret_cast<double*>(tw + M);
  float2* Pb = reinterpret_cast<float2*>(red + F::NRED);  // [K][M][W]
  float* slot = reinterpret_cast<float*>(Pb + K * M * F::W);  // [0] probe max, [1] object max
  float* redf = reinterpret_cast<float*>(red);
  const int tid = threadIdx.x;
  const int c = (C > 1) ? (int)(blockIdx.x % C) : 0;

  FourierArgs fa;
  fa.amp = a.amp;
  fa.amp_scale = a.amp_scale;
  fa.istore = a.istore;

  for (int i = tid; i < M; i += F::NT) tw[i] = a.tw[i];
  for (int e = tid; e < K * M * F::W; e += F::NT) {
    const int colL = e % F::W, row = (e / F::W) % M, k = e / (F::W * M);
    Pb[e] = a.P[((size_t)k * M + row) * M + c * F::W + colL];
  }
  __syncthreads();

  for (int it = 0; it < a.n_iter; ++it) {
    const bool upd = (a.t0 + it) >= (long long)a.probe_start;
    for (int s = 0; s < a.J; ++s) {
      const int j = a.order[(size_t)it * a.J + s];
      const int2 p = a.pos[j];
      // prologue: exit waves into layout A, local maxima of sum_k|P_k|^2 and |O_j|^2
      float pm = 0.f, om = 0.f;
      for (int e = tid; e < M * F::W; e += F::NT) {
        const int colL = e % F::W, row = e / F::W;
        const float2 o = __ldcg(a.O + (size_t)(p.x + row) * a.nx + p.y + c * F::W + colL);
        om = fmaxf(om, cabs2(o));
        float ps = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const float2 pr = Pb[(k * M + row) * F::W + colL];
          ps += cabs2(pr);
          buf[k * M * F::PA + row * F::PA + colL] = cmul(pr, o);
        }
        pm = fmaxf(pm, ps);
      }
      pm = block_max_f<F::NT>(pm, redf);
      om = block_max_f<F::NT>(om, redf + 32);
      if (tid == 0) {
        slot[0] = pm;
        slot[1] = om;
      }
      __syncthreads();
      fft_lines<M, F::E, K * F::W, F::W, M * F::PA, 1, F::PA, F::NT, false>(buf, tw);
      float pmax, omax;
      if constexpr (C > 1) {
        cg::cluster_group cl = cg::this_cluster();
        cl.sync();  // layout A and the maxima slots are visible cluster-wide
        pmax = 0.f;
        omax = 0.f;
#pragma unroll
        for (int r = 0; r < C; ++r) {
          const float* rs = cl.map_shared_rank(slot, r);
          pmax = fmaxf(pmax, rs[0]);
          omax = fmaxf(omax, rs[1]);
        }
        transpose_A_to_B<F, false>(buf, c);
      } else {
        pmax = slot[0];
        omax = slot[1];
      }
      fft_lines<M, F::E, K * F::H, K * F::H, 0, F::PB, 1, F::NT, false>(buf, tw);
      project_difference<F>(buf, fa, j, c);
      fft2_inverse<F>(buf, tw, c);

      // update of this CTA's columns of O_j and of the probe
      const float sa = pmax > 0.f ? a.alpha / pmax : 0.f;
      const float sb = (upd && omax > 0.f) ? a.beta / omax : 0.f;
      for (int e = tid; e < M * F::W; e += F::NT) {
        const int colL = e % F::W, row = e / F::W;
        float2* op = a.O + (size_t)(p.x + row) * a.nx + p.y + c * F::W + colL;
        const float2 o = __ldcg(op);
        float2 num = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const float2 d = buf[k * M * F::PA + row * F::PA + colL];
          float2& pr = Pb[(k * M + row) * F::W + colL];
          num = cadd(num, cconjmul(pr, d));
          if (upd) pr = cadd(pr, cscale(cconjmul(o, d), sb));
        }
        __stcg(op, cadd(o, cscale(num, sa)));
      }
      if constexpr (C > 1) cg::this_cluster().sync();
      else __syncthreads();
    }
  }
  for (int e = tid; e < K * M * F::W; e += F::NT) {
    const int colL = e % F::W, row = (e / F::W) % M, k = e / (F::W * M);
    a.P[((size_t)k * M + row) * M + c * F::W + colL] = Pb[e];
  }
}

}  // namespace ptycho

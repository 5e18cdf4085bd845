// ePIE sweep (Maiden & Rodenburg 2009; multi-mode probe, Thibault & Menzel
// 2013) as one persistent thread-block cluster, with the register-resident
// transforms and asynchronous transposes of k_fourier3.
//
// ePIE is sequential: each position's update feeds the next, so the sweep is
// bound by the latency of one position, not by bandwidth.  Per position j
// (values from before this position's update):
//   psi_k = P_k O_j;  Delta_k = F^-1 Pi(F psi)_k - psi_k
//   O_j  += alpha sum_k conj(P_k) Delta_k / max_u sum_k |P_k(u)|^2
//   P_k  += beta conj(O_j) Delta_k / max_u |O_j(u)|^2      (t >= probe_start)
//
// CTA c of the cluster owns columns [c W, (c+1) W) of the patch, and so the
// same columns of every probe mode for the whole launch (shared memory, exact
// FP32, written back at the end).  The object stays in global memory (L2);
// it is read and written with L2-coherent (.cg) accesses.
//
// Per position: prologue (P O into registers, the CTA's maxima), column
// stages, transpose into the peers' row buffers with st.async completing on
// their mbarriers -- the same messages carry each CTA's two maxima, so the
// cluster-wide maxima arrive with the data --, row stages, projection,
// inverse row stages, transpose back, inverse column stages, the update of
// the CTA's columns, and one cluster barrier (release / acquire) that makes
// the object writes visible before the next position reads them.  The
// barrier also orders the reuse of the row buffer, the maxima inbox and the
// mbarrier phases: a peer sends the next position's data only after it.
#pragma once
#include "fourier3.cuh"

namespace ptycho {

struct Epie2Args {
  float2* O;              // object [ny][nx] (in/out)
  int nx;
  float2* P;              // probe [K][M][M] (in/out)
  const int2* pos;        // [J]
  const void* amp;        // sqrt(I) in FFT order [J][M][M]
  const float* amp_scale;
  int istore;
  const float2* tw2;      // tw2[k1 * R2 + n2] = exp(-2 pi i n2 k1 / M)
  const int* order;       // [n_iter][J] visiting order
  int J, n_iter;
  long long t0;           // iteration index of the first iteration
  int probe_start;
  float alpha, beta;
  int* err_flag;
};

// bytes of dynamic shared memory: column buffer X, row buffer Y, probe
// columns, twiddle tables, maxima inbox [C], reduction scratch, mbarriers
template <class F>
__host__ __device__ constexpr size_t epie2_smem() {
  return (size_t)F::L * 8 + (size_t)F::K * F::H * F::PB * 8 + (size_t)F::L * 8 + (size_t)F::M * 16 +
         (size_t)F::C * 8 + 64 * 4 + 16;
}

// Bounded wait on phase `parity` of an mbarrier (see mbar_wait0_or_abort).
__device__ __forceinline__ bool mbar_wait_parity_or_abort(uint64_t* bar, uint32_t parity, const int* err_flag) {
  uint32_t done = 0;
  for (int i = 0; i < (1 << 20) && !done; ++i) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (!done && (i & 255) == 255 && *(volatile const int*)err_flag) break;
  }
  return done != 0;
}

template <int M, int K, int C>
__global__ void __launch_bounds__(F2<M, K, C>::NT, 1) k_epie2(Epie2Args a) {
  using F = F2<M, K, C>;
  static_assert(C > 1, "cluster kernel");
  constexpr int R1 = F::R1, R2 = F::R2, W = F::W, H = F::H, NT = F::NT, Q = F::Q;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* X = reinterpret_cast<float2*>(smem_raw);  // column layout, cb<F>()
  float2* Y = X + F::L;                               // row layout, rb<F>()
  float2* Pb = Y + K * H * F::PB;                     // probe columns, cb<F>() layout
  float2* tw = Pb + F::L;
  float2* twT = tw + M;
  float2* mx = twT + M;                               // maxima inbox: (pmax, omax) of each CTA
  float* redf = reinterpret_cast<float*>(mx + C);
  uint64_t* barY = reinterpret_cast<uint64_t*>(redf + 64);
  uint64_t* barX = barY + 1;

  const int tid = threadIdx.x;
  const int c = (int)(blockIdx.x % C);
  constexpr uint32_t BYTES_Y = K * H * M * 8 + C * 8;  // row data + one maxima pair per CTA
  constexpr uint32_t BYTES_X = K * M * W * 8;

  if (tid == 0) {
    mbar_init(barY, 1);
    mbar_init(barX, 1);
  }
  for (int i = tid; i < M; i += NT) {
    const float2 t = a.tw2[i];
    tw[i] = t;
    twT[(i % R2) * R1 + i / R2] = t;
  }
  for (int e = tid; e < F::L; e += NT) {
    const int colL = e % W, row = (e / W) % M, k = e / (W * M);
    Pb[cb<F>(k, row, colL)] = a.P[((size_t)k * M + row) * M + c * W + colL];
  }
  // barriers initialised and probe columns loaded before any peer signals
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
  constexpr float inv = 1.0f / (float)(M * M);
  uint32_t phase = 0;
  // this thread's part of max_u sum_k |P_k(u)|^2 for the next position:
  // computed by the probe update (or unchanged without one); < 0 = not yet
  float pm_next = -1.f;

  for (int it = 0; it < a.n_iter; ++it) {
    const bool upd = (a.t0 + it) >= (long long)a.probe_start;
    for (int s = 0; s < a.J; ++s, phase ^= 1u) {
      const int j = a.order[(size_t)it * a.J + s];
      const int2 p = a.pos[j];
      const size_t amp_row0 = ((size_t)j * M + c * H) * M;
      if (tid == 0) {
        mbar_expect(barY, BYTES_Y);
        mbar_expect(barX, BYTES_X);
        const size_t esz = a.istore == 0 ? 4 : 2;
        prefetch_l2(reinterpret_cast<const unsigned char*>(a.amp) + amp_row0 * esz, (uint32_t)(H * M * esz));
      }
      // ---- prologue: psi = P_k O_j in registers, this CTA's maxima
      float2 v[R1];
      float om = 0.f, pm = 0.f;
      {
        const int colL = tid % W, n2 = (tid / W) % R2, k = tid / (W * R2);
        const float2* orow = a.O + (size_t)(p.x + n2) * a.nx + p.y + c * W + colL;
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) {
          const float2 o = __ldcg(orow + (size_t)n1 * R2 * a.nx);
          om = fmaxf(om, cabs2(o));
          const float2 z = cmul(Pb[cb<F>(k, n1 * R2 + n2, colL)], o);
          v[n1] = z;
        }
      }
      if (pm_next >= 0.f) {
        pm = pm_next;
      } else {
        for (int e = tid; e < M * W; e += NT) {
          float ps = 0.f;
#pragma unroll
          for (int k = 0; k < K; ++k) ps += cabs2(Pb[k * M * W + e]);
          pm = fmaxf(pm, ps);
        }
      }
      const float pm_own = pm;
      // both CTA maxima in one block reduction (valid in thread 0, which
      // sends them to the peers)
      {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          pm = fmaxf(pm, __shfl_down_sync(0xffffffffu, pm, o));
          om = fmaxf(om, __shfl_down_sync(0xffffffffu, om, o));
        }
        constexpr int NW = (NT + 31) / 32;
        const int lane = tid & 31, wid = tid >> 5;
        __syncthreads();
        if (lane == 0) {
          redf[wid] = pm;
          redf[32 + wid] = om;
        }
        __syncthreads();
        if (tid == 0)
          for (int i = 1; i < NW; ++i) {
            pm = fmaxf(pm, redf[i]);
            om = fmaxf(om, redf[32 + i]);
          }
      }
      // ---- column stage 1
      {
        const int colL = tid % W, n2 = (tid / W) % R2, k = tid / (W * R2);
        dft<R1, false>(v);
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1) v[k1] = cmul(v[k1], tw[k1 * R2 + n2]);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) X[cb<F>(k, k1 * R2 + n2, colL)] = v[k1];
      }
      __syncthreads();
      // ---- column stage 2 -> peers' row buffers (and this CTA's maxima)
      {
        float2 w[Q][R2];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int s2 = tid + q * NT;
          const int colL = s2 % W, k1 = (s2 / W) % R1, k = s2 / (W * R1);
#pragma unroll
          for (int n2 = 0; n2 < R2; ++n2) w[q][n2] = X[cb<F>(k, k1 * R2 + n2, colL)];
          dft<R2, false>(w[q]);
        }
        const uint32_t barY_l = smem_u32(barY);
        if (tid == 0) {
          const float2 mine = make_float2(pm, om);
          for (int r = 0; r < C; ++r)
            st_async_f2(mapa_u32(smem_u32(mx + c), (uint32_t)r), mine, mapa_u32(barY_l, (uint32_t)r));
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int s2 = tid + q * NT;
          const int colL = s2 % W, k1 = (s2 / W) % R1, k = s2 / (W * R1);
          const int col = c * W + colL;
#pragma unroll
          for (int k2 = 0; k2 < R2; ++k2) {
            const int f = k1 + R1 * k2;
            const uint32_t rank = (uint32_t)(f / H);
            st_async_f2(mapa_u32(smem_u32(Y + rb<F>(k, f % H, col)), rank), w[q][k2], mapa_u32(barY_l, rank));
          }
        }
      }
      const float scale = a.istore != 0 ? __ldg(a.amp_scale + j) : 1.f;
      // this thread's amplitudes for the projection, loaded while the
      // transpose completes (K = 1: in the register layout of row stage 2)
      constexpr int NA = (H * M + NT - 1) / NT;
      float amv[K > 1 ? NA : 1];
      float am1[K == 1 ? Q : 1][K == 1 ? R2 : 1];
      if constexpr (K == 1) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int s2 = tid + q * NT;
          const int k1 = s2 % R1, rowL = (s2 / R1) % H;
#pragma unroll
          for (int k2 = 0; k2 < R2; ++k2) {
            const size_t ai = amp_row0 + (size_t)rowL * M + k1 + R1 * k2;
            float am;
            if (a.istore == 0) am = __ldcg(reinterpret_cast<const float*>(a.amp) + ai);
            else if (a.istore == 1) am = __half2float(reinterpret_cast<const __half*>(a.amp)[ai]) * scale;
            else am = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(a.amp)[ai]) * scale;
            am1[q][k2] = am;
          }
        }
      } else {
#pragma unroll
        for (int q = 0; q < NA; ++q) {
          const int px = tid + q * NT;
          if (px < H * M) {
            const int rowL = px / M, pp = px % M;
            const size_t ai = amp_row0 + (size_t)rowL * M + pp / R2 + R1 * (pp % R2);
            if (a.istore == 0) amv[q] = __ldcg(reinterpret_cast<const float*>(a.amp) + ai);
            else if (a.istore == 1) amv[q] = __half2float(reinterpret_cast<const __half*>(a.amp)[ai]) * scale;
            else amv[q] = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(a.amp)[ai]) * scale;
          }
        }
      }
      if (!mbar_wait_parity_or_abort(barY, phase, a.err_flag)) atomicExch(a.err_flag, 1);
      // ---- row stage 1
      {
        const int n2 = tid % R2, rowL = (tid / R2) % H, k = tid / (R2 * H);
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) v[n1] = Y[rb<F>(k, rowL, n1 * R2 + n2)];
        dft<R1, false>(v);
#pragma unroll
        for (int k1 = 1; k1 < R1; ++k1) v[k1] = cmul(v[k1], tw[k1 * R2 + n2]);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) Y[rb<F>(k, rowL, k1 * R2 + n2)] = v[k1];
      }
      __syncthreads();
      // ---- row stage 2, projection (modes summed through shared memory for
      // K > 1), first inverse stage
      {
        float2 w[Q][R2];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int s2 = tid + q * NT;
          const int k1 = s2 % R1, rowL = (s2 / R1) % H, k = s2 / (R1 * H);
#pragma unroll
          for (int n2 = 0; n2 < R2; ++n2) w[q][n2] = Y[rb<F>(k, rowL, k1 * R2 + n2)];
          dft<R2, false>(w[q]);
        }
        if constexpr (K == 1) {
#pragma unroll
          for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2)
              w[q][k2] = cscale(w[q][k2], proj_factor(FM_CHI, am1[q][k2], cabs2(w[q][k2])) * inv);
        } else {
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            const int s2 = tid + q * NT;
            const int k1 = s2 % R1, rowL = (s2 / R1) % H, k = s2 / (R1 * H);
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) Y[rb<F>(k, rowL, k1 * R2 + k2)] = w[q][k2];
          }
          __syncthreads();
#pragma unroll
          for (int q = 0; q < NA; ++q) {
            const int px = tid + q * NT;
            if (px >= H * M) continue;
            const int rowL = px / M, pp = px % M;  // pp = k1 * R2 + k2 storage slot
            float2 z[K];
            float A2 = 0.f;
#pragma unroll
            for (int k = 0; k < K; ++k) {
              z[k] = Y[rb<F>(k, rowL, pp)];
              A2 += cabs2(z[k]);
            }
            const float fct = proj_factor(FM_CHI, amv[q], A2) * inv;
#pragma unroll
            for (int k = 0; k < K; ++k) Y[rb<F>(k, rowL, pp)] = cscale(z[k], fct);
          }
          __syncthreads();
#pragma unroll
          for (int q = 0; q < Q; ++q) {
            const int s2 = tid + q * NT;
            const int k1 = s2 % R1, rowL = (s2 / R1) % H, k = s2 / (R1 * H);
#pragma unroll
            for (int k2 = 0; k2 < R2; ++k2) w[q][k2] = Y[rb<F>(k, rowL, k1 * R2 + k2)];
          }
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int s2 = tid + q * NT;
          const int k1 = s2 % R1;
          dft<R2, true>(w[q]);
#pragma unroll
          for (int n2 = 1; n2 < R2; ++n2) w[q][n2] = cmul(w[q][n2], cconj(twT[n2 * R1 + k1]));
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int s2 = tid + q * NT;
          const int k1 = s2 % R1, rowL = (s2 / R1) % H, k = s2 / (R1 * H);
#pragma unroll
          for (int n2 = 0; n2 < R2; ++n2) Y[rb<F>(k, rowL, k1 * R2 + n2)] = w[q][n2];
        }
      }
      __syncthreads();
      // ---- inverse row stage B -> peers' column buffers
      {
        const int n2 = tid % R2, rowL = (tid / R2) % H, k = tid / (R2 * H);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) v[k1] = Y[rb<F>(k, rowL, k1 * R2 + n2)];
        dft<R1, true>(v);
        const int f = c * H + rowL;
        const uint32_t barX_l = smem_u32(barX);
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) {
          const int x = n1 * R2 + n2;
          const uint32_t rank = (uint32_t)(x / W);
          st_async_f2(mapa_u32(smem_u32(X + cb<F>(k, f, x % W)), rank), v[n1], mapa_u32(barX_l, rank));
        }
      }
      if (!mbar_wait_parity_or_abort(barX, phase, a.err_flag)) atomicExch(a.err_flag, 1);
      // ---- inverse column stage A
      {
        float2 w[Q][R2];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int s2 = tid + q * NT;
          const int colL = s2 % W, k1 = (s2 / W) % R1, k = s2 / (W * R1);
#pragma unroll
          for (int k2 = 0; k2 < R2; ++k2) w[q][k2] = X[cb<F>(k, k1 + R1 * k2, colL)];
          dft<R2, true>(w[q]);
#pragma unroll
          for (int n2 = 0; n2 < R2; ++n2) w[q][n2] = cmul(w[q][n2], cconj(tw[k1 * R2 + n2]));
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int s2 = tid + q * NT;
          const int colL = s2 % W, k1 = (s2 / W) % R1, k = s2 / (W * R1);
#pragma unroll
          for (int n2 = 0; n2 < R2; ++n2) X[cb<F>(k, k1 + R1 * n2, colL)] = w[q][n2];
        }
      }
      __syncthreads();
      // ---- inverse column stage B: Delta_k into X (rows n1*R2 + n2)
      {
        const int colL = tid % W, n2 = (tid / W) % R2, k = tid / (W * R2);
#pragma unroll
        for (int k1 = 0; k1 < R1; ++k1) v[k1] = X[cb<F>(k, k1 + R1 * n2, colL)];
        dft<R1, true>(v);
        __syncthreads();  // every thread has read its inputs before X is reused
#pragma unroll
        for (int n1 = 0; n1 < R1; ++n1) X[cb<F>(k, n1 * R2 + n2, colL)] = v[n1];
      }
      __syncthreads();
      // ---- update of this CTA's columns of O_j and of the probe
      {
        float pmax = 0.f, omax = 0.f;
#pragma unroll
        for (int r = 0; r < C; ++r) {
          pmax = fmaxf(pmax, mx[r].x);
          omax = fmaxf(omax, mx[r].y);
        }
        const float sa = pmax > 0.f ? a.alpha / pmax : 0.f;
        const float sb = (upd && omax > 0.f) ? a.beta / omax : 0.f;
        // all of this thread's object values in flight first (the loop
        // otherwise waits for one L2 round trip per element)
        constexpr int NU = (M * W + NT - 1) / NT;
        float2 ov[NU];
#pragma unroll
        for (int q = 0; q < NU; ++q) {
          const int e = tid + q * NT;
          if (e < M * W) ov[q] = __ldcg(a.O + (size_t)(p.x + e / W) * a.nx + p.y + c * W + e % W);
        }
        float pmx = 0.f;
#pragma unroll
        for (int q = 0; q < NU; ++q) {
          const int e = tid + q * NT;
          if (e >= M * W) continue;
          const int colL = e % W, row = e / W;
          const float2 o = ov[q];
          float2 num = make_float2(0.f, 0.f);
          float ps = 0.f;
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const float2 d = X[cb<F>(k, row, colL)];
            float2& pr = Pb[cb<F>(k, row, colL)];
            num = cadd(num, cconjmul(pr, d));
            if (upd) {
              pr = cadd(pr, cscale(cconjmul(o, d), sb));
              ps += cabs2(pr);
            }
          }
          pmx = fmaxf(pmx, ps);
          __stcg(a.O + (size_t)(p.x + row) * a.nx + p.y + c * W + colL, cadd(o, cscale(num, sa)));
        }
        pm_next = upd ? pmx : pm_own;
      }
      // object writes visible cluster-wide; buffers and barriers free for the
      // next position
      asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    }
  }
  for (int e = tid; e < F::L; e += NT) {
    const int colL = e % W, row = (e / W) % M, k = e / (W * M);
    a.P[((size_t)k * M + row) * M + c * W + colL] = Pb[cb<F>(k, row, colL)];
  }
}

}  // namespace ptycho

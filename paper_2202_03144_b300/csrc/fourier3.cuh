// Fused Fourier step, cluster form with asynchronous transposes.
//
// Same transforms, task mapping and arithmetic as k_fourier2 (two register
// radix stages per 1-D transform, modulus projection between the forward and
// the inverse transform), but the two cluster-wide transposes are
// asynchronous stores into the peer CTA's shared memory that complete a
// transaction count on the peer's mbarrier (st.async ... complete_tx):
//
//   * separate column (X) and row (Y) buffers, so no CTA overwrites data a
//     peer is still reading: the write-after-read cluster barriers of
//     k_fourier2 are gone;
//   * a receiver waits only on its own mbarrier for the bytes it expects
//     (K*H*M*8 into Y, K*M*W*8 into X): no release/acquire cluster barrier
//     and no memory fence per transpose;
//   * one split cluster barrier at the start (arrive after the mbarriers are
//     initialised, wait just before the first remote store) keeps a fast CTA
//     from signalling a peer's barrier before it exists.
//
// Ordering of the reuse of X: a CTA reads its X in column stage 2 and only
// then sends its first-transpose data; a peer writes into this X in the
// second transpose only after it has received that data, so the reads are
// done.  Every write into a CTA's shared memory is counted by its mbarriers
// and waited for before the CTA exits.
//
// The amplitudes sqrt(I) are prefetched into L2 at kernel start (one bulk
// prefetch per CTA) and read into registers while the first transpose
// completes; the
// shared memory saved (two 32 KB buffers instead of one plus a 16 KB
// amplitude tile and the barriers) keeps three 256-thread CTAs per SM at
// M = 256, C = 16.
#pragma once
#include "fourier2.cuh"

namespace ptycho {

// Merged column and row buffer (the DM pass of the one-mode 256^2 shapes):
// one 32 KB exchange buffer instead of two, so four CTAs share an SM (at 64
// registers); the two write-after-read hazards that separate buffers avoid
// -- a peer still reading its buffer when this CTA's transpose data arrives
// in it -- are closed by a split cluster barrier before each transpose
// (arrive once a thread has consumed what it read from the buffer, wait
// with acquire just before its first remote store).  Measured at 256^2 x 10k
// positions: DM pass 7.10 against 7.92 ms with two buffers (it also streams
// psi, and the fourth CTA hides that latency); the LSQML residual pass
// loses (6.25 against 6.07 ms), so it keeps two buffers unless
// PT_F3_MERGED_CHI is set.
#ifndef PT_F3_MERGED_CHI
#define PT_F3_MERGED_CHI 0
#endif
// 1 (default): the merged form arrives (relaxed) after the radix stage has
// consumed the values it read -- the reads are then complete, so no release
// fence is needed; 0: it arrives (release) right after issuing the reads.
// DM pass at 256^2 x 10k: 7.10 against 7.40 ms.
#ifndef PT_F3_ARRIVE_LATE
#define PT_F3_ARRIVE_LATE 1
#endif
template <class F, int MODE_T>
__host__ __device__ constexpr bool f3_merged() {
  return (MODE_T == FM_DM || (PT_F3_MERGED_CHI && MODE_T == FM_CHI)) && F::K == 1 && F::M == 256 &&
         F::L == F::K * F::H * F::PB;
}

// bytes of dynamic shared memory: X, Y (one buffer when merged), twiddle
// tables, reduction scratch, two mbarriers
template <class F, int MODE_T = -1>
__host__ __device__ constexpr size_t fourier3_smem() {
  return (size_t)F::L * 8 + (f3_merged<F, MODE_T>() ? 0 : (size_t)F::K * F::H * F::PB * 8) + (size_t)F::M * 16 +
         F::NRED * 8 + 16;
}

__device__ __forceinline__ void st_async_f2(uint32_t addr, float2 v, uint32_t bar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(addr),
               "f"(v.x), "f"(v.y), "r"(bar)
               : "memory");
}
__device__ __forceinline__ void mbar_expect(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// Bounded wait for the completion of phase 0 of a transpose barrier.  After
// `limit` polls (the context's wait limit; 0 gives up at once) the wait
// raises the error flag and keeps waiting, now with a fixed bound: the peers'
// stores into this CTA's shared memory are on their way (every CTA sends its
// transpose data unconditionally), and none may land after the buffer has
// been reused or the CTA has exited.  Only if the data is still missing after
// the fixed bound does the CTA go on without it.
__device__ __forceinline__ void mbar_wait_flag(uint64_t* bar, int* err_flag, int limit) {
  uint32_t done = 0;
  for (int i = 0; i < limit && !done; ++i)
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar))
        : "memory");
  if (done) return;
  atomicExch(err_flag, 1);
  for (int i = 0; i < (1 << 22) && !done; ++i)
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar))
        : "memory");
}

template <int IST>
__device__ __forceinline__ float amp_global(const Fourier2Args& a, size_t idx, float scale) {
  const int ist = IST >= 0 ? IST : a.istore;
  if (ist == 0) return __ldcs(reinterpret_cast<const float*>(a.amp) + idx);
  const unsigned short u = __ldcs(reinterpret_cast<const unsigned short*>(a.amp) + idx);
  if (ist == 1) return __half2float(__ushort_as_half(u)) * scale;
  return __bfloat162float(__ushort_as_bfloat16(u)) * scale;
}

// object loads in flight per thread in the prologue (4 and 8 measured equal)
#ifndef PT_F3_OG
#define PT_F3_OG 4
#endif
constexpr int F3_OG = PT_F3_OG;

// CTAs per SM for the launch bounds: by threads (and the radix-24 register
// demand) and by shared memory
// CTAs per SM asked of shapes with at most 128 threads per CTA (128^2 on
// 8-CTA clusters): 6 for the LSQML residual pass (117 -> 80 registers:
// 1.19 -> 1.09 ms per 10k positions), 5 for the DM pass (1.37 -> 1.30 ms; at
// 6 it loses half of that), 0 = the default rule (3)
#ifndef PT_F3_MINB_NT128
#define PT_F3_MINB_NT128 0
#endif
template <class F, int MODE_T>
constexpr int f3_min_blocks() {
  const int nt128 = PT_F3_MINB_NT128 > 0 ? PT_F3_MINB_NT128 : (MODE_T == FM_DM ? 5 : 6);
  const int by_threads = F::R1 > 16 ? 1
                                    : (F::NT <= 128 ? nt128
                                                    : (F::NT <= 256 ? (f3_merged<F, MODE_T>() ? 4 : 3) : (F::NT <= 512 ? 2 : 1)));
  const int by_smem = (int)((228 * 1024) / (fourier3_smem<F, MODE_T>() + 1024));
  const int b = by_threads < by_smem ? by_threads : by_smem;
  return b < 1 ? 1 : b;
}

template <int M, int K, int C, int MODE_T = -1, int IST_T = -1>
__global__ void __launch_bounds__(F2<M, K, C>::NT, f3_min_blocks<F2<M, K, C>, MODE_T>()) k_fourier3(Fourier2Args a) {
  using F = F2<M, K, C>;
  static_assert(C > 1, "cluster kernel");
  constexpr int R1 = F::R1, R2 = F::R2, W = F::W, H = F::H, NT = F::NT, Q = F::Q;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr bool MERGED = f3_merged<F, MODE_T>();
  float2* X = reinterpret_cast<float2*>(smem_raw);  // column layout, cb<F>()
  float2* Y = MERGED ? X : X + F::L;                  // row layout, rb<F>()
  float2* tw = X + F::L + (MERGED ? 0 : K * H * F::PB);  // tw[k1 * R2 + n2] = W_M^(n2 k1)
  float2* twT = tw + M;                               // twT[n2 * R1 + k1]
  double* red = reinterpret_cast<double*>(twT + M);
  uint64_t* barY = reinterpret_cast<uint64_t*>(red + F::NRED);
  uint64_t* barX = barY + 1;

  pdl_wait();
  pdl_launch();
  const int tid = threadIdx.x;
  const int c = (int)(blockIdx.x % C);
  const int j = a.j0 + (int)(blockIdx.x / C);
  // probe of this position (sub-pixel: its bin of the shifted-probe table)
  const float2* Pj = a.pbin ? a.P + (size_t)__ldg(a.pbin + j) * (K * M * M) : a.P;
  const int mode = MODE_T >= 0 ? MODE_T : a.mode;
  const int istore = IST_T >= 0 ? IST_T : a.istore;
  const int2 p = a.pos[j];
  const bool need_amp = mode != FM_SIM;
  const size_t amp_row0 = ((size_t)j * M + c * H) * M;  // first amplitude of this CTA's rows

  if (tid == 0) {
    mbar_init(barY, 1);
    mbar_init(barX, 1);
    mbar_expect(barY, (uint32_t)(K * H * M * 8));
    mbar_expect(barX, (uint32_t)(K * M * W * 8));
    if (need_amp) {
      const size_t esz = istore == 0 ? 4 : 2;
      prefetch_l2(reinterpret_cast<const unsigned char*>(a.amp) + amp_row0 * esz, (uint32_t)(H * M * esz));
    }
  }
  // barriers initialised: peers may signal them once they pass the wait below
  // (merged buffer: the arrive after column stage 2's reads does this too)
  if (!MERGED) asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
  for (int i = tid; i < M; i += NT) {
    const float2 t = a.tw2[i];
    tw[i] = t;
    twT[(i % R2) * R1 + i / R2] = t;
  }

  float2 v[R1];
  // ---- prologue + column stage 1: thread = (k, colL, n2), rows n1*R2 + n2
  {
    const int colL = tid % W, n2 = (tid / W) % R2, k = tid / (W * R2);
    const int col = c * W + colL;
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) v[n1] = __ldg(Pj + ((size_t)k * M + n1 * R2 + n2) * M + col);
    const float2* orow = a.O + (size_t)(p.x + n2) * a.nx + p.y + col;
#pragma unroll
    for (int g0 = 0; g0 < R1; g0 += F3_OG) {
      float2 o[F3_OG];
#pragma unroll
      for (int i = 0; i < F3_OG && g0 + i < R1; ++i) o[i] = __ldg(orow + (size_t)(g0 + i) * R2 * a.nx);
#pragma unroll
      for (int i = 0; i < F3_OG && g0 + i < R1; ++i) v[g0 + i] = cmul(v[g0 + i], o[i]);
      asm volatile("" ::: "memory");
    }
    if (mode == FM_DM) {
      const float2* xrow = a.X + (((size_t)(j - a.xoff) * K + k) * M + n2) * M + col;
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) v[n1] = csub(cscale(v[n1], 2.f), xrow[(size_t)n1 * R2 * M]);
    }
    __syncthreads();  // twiddle table
    dft<R1, false>(v);
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) v[k1] = cmul(v[k1], tw[k1 * R2 + n2]);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) X[cb<F>(k, k1 * R2 + n2, colL)] = v[k1];
  }
  __syncthreads();
  // ---- column stage 2: task (k, colL, k1) -> frequency rows k1 + R1*k2,
  // stored asynchronously into row buffer Y of the CTA owning each row
  {
    float2 w[Q][R2];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int s = tid + q * NT;
      const int colL = s % W, k1 = (s / W) % R1, k = s / (W * R1);
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) w[q][n2] = X[cb<F>(k, k1 * R2 + n2, colL)];
      // merged: this thread's reads of the buffer are issued; peers may
      // overwrite it (with their row data) once every thread has arrived
      if (MERGED && !PT_F3_ARRIVE_LATE && q == Q - 1)
        asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
      dft<R2, false>(w[q]);
    }
    // (late form: the values are consumed, so the reads are complete)
    if (MERGED && PT_F3_ARRIVE_LATE) asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
    // peers' barriers exist (and, merged, every peer has read its buffer)
    if (MERGED) asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
    else asm volatile("barrier.cluster.wait.aligned;" ::: "memory");
    const uint32_t barY_l = smem_u32(barY);
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int s = tid + q * NT;
      const int colL = s % W, k1 = (s / W) % R1, k = s / (W * R1);
      const int col = c * W + colL;
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) {
        const int f = k1 + R1 * k2;
        const uint32_t rank = (uint32_t)(f / H);
        st_async_f2(mapa_u32(smem_u32(Y + rb<F>(k, f % H, col)), rank), w[q][k2], mapa_u32(barY_l, rank));
      }
    }
  }
  // this thread's amplitudes for row stage 2 (K = 1: the projection runs in
  // registers)
  float scale = 1.f;
  if (need_amp && istore != 0) scale = __ldg(a.amp_scale + j);
  float am[Q][R2];
  auto load_amp = [&]() {
    if (K == 1 && need_amp) {
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int s = tid + q * NT;
        const int k1 = s % R1, rowL = (s / R1) % H;
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2)
          am[q][k2] = amp_global<IST_T>(a, amp_row0 + (size_t)rowL * M + k1 + R1 * k2, scale);
      }
    }
  };
  // K > 1: the amplitudes of this thread's pixels in the mode-summing loop
  // below, all loads in flight at once
  constexpr int NA = (H * M + NT - 1) / NT;
  float amv[K > 1 ? NA : 1];
  auto load_amp_k = [&]() {
    if constexpr (K > 1) {
      if (need_amp) {
#pragma unroll
        for (int q = 0; q < NA; ++q) {
          const int px = tid + q * NT;
          if (px < H * M) {
            const int rowL = px / M, pp = px % M;
            amv[q] = amp_global<IST_T>(a, amp_row0 + (size_t)rowL * M + pp / R2 + R1 * (pp % R2), scale);
          }
        }
      }
    }
  };
  // LSQML residual pass: before the wait (256^2: 6.51 -> 6.24 ms); DM pass,
  // whose prologue holds more registers: after row stage 1 (2% faster there)
  constexpr bool amp_early = MODE_T != FM_DM && !MERGED;
  if (amp_early) {
    load_amp();
    load_amp_k();
  }
  mbar_wait_flag(barY, a.err_flag, a.wait_limit);
  // ---- row stage 1: task (k, rowL, n2'), columns n1'*R2 + n2'
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
  if (!amp_early) {
    load_amp();
    load_amp_k();
  }
  __syncthreads();
  // ---- row stage 2 (+ projection + first inverse stage)
  constexpr float inv = 1.0f / (float)(M * M);
  // Fourier error: per-thread FP32 partials over the thread's few dozen pixels
  // (A - a is exact in FP32 where A and a are within a factor 2), FP64 from the
  // block sums on
  float en = 0.f, ed = 0.f;
  {
    float2 w[Q][R2];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int s = tid + q * NT;
      const int k1 = s % R1, rowL = (s / R1) % H, k = s / (R1 * H);
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) w[q][n2] = Y[rb<F>(k, rowL, k1 * R2 + n2)];
      dft<R2, false>(w[q]);
      if constexpr (K == 1) {
        const int ky = c * H + rowL;
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
          const int kx = k1 + R1 * k2;
          const float A2 = cabs2(w[q][k2]);
          if (mode == FM_SIM) {
            a.I_out[((size_t)j * M + ((ky + M / 2) % M)) * M + ((kx + M / 2) % M)] = A2;
          } else if (mode == FM_ERR) {
            if (am[q][k2] >= 0.f) {
              const float d = sqrtf(A2) - am[q][k2];
              en = fmaf(d, d, en);
              ed = fmaf(am[q][k2], am[q][k2], ed);
            }
          } else {
            const float fct = proj_factor(mode, am[q][k2], A2);
            w[q][k2] = cscale(w[q][k2], fct * inv);
          }
        }
      }
    }
    if constexpr (K > 1) {
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int s = tid + q * NT;
        const int k1 = s % R1, rowL = (s / R1) % H, k = s / (R1 * H);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) Y[rb<F>(k, rowL, k1 * R2 + k2)] = w[q][k2];
      }
      __syncthreads();
#pragma unroll
      for (int q = 0; q < NA; ++q) {
        const int px = tid + q * NT;
        if (px >= H * M) continue;
        const int rowL = px / M, pp = px % M;
        const int kx = pp / R2 + R1 * (pp % R2);
        const int ky = c * H + rowL;
        float2 z[K];
        float A2 = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          z[k] = Y[rb<F>(k, rowL, pp)];
          A2 += cabs2(z[k]);
        }
        if (mode == FM_SIM) {
          a.I_out[((size_t)j * M + ((ky + M / 2) % M)) * M + ((kx + M / 2) % M)] = A2;
          continue;
        }
        const float am = amv[q];
        if (mode == FM_ERR) {
          if (am >= 0.f) {
            const float d = sqrtf(A2) - am;
            en = fmaf(d, d, en);
            ed = fmaf(am, am, ed);
          }
          continue;
        }
        const float fct = proj_factor(mode, am, A2);
#pragma unroll
        for (int k = 0; k < K; ++k) Y[rb<F>(k, rowL, pp)] = cscale(z[k], fct * inv);
      }
      __syncthreads();
      if (mode == FM_DM || mode == FM_CHI || mode == FM_CHIP) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int s = tid + q * NT;
          const int k1 = s % R1, rowL = (s / R1) % H, k = s / (R1 * H);
#pragma unroll
          for (int k2 = 0; k2 < R2; ++k2) w[q][k2] = Y[rb<F>(k, rowL, k1 * R2 + k2)];
        }
      }
    }
    if (mode == FM_ERR) {
      const double sn = block_sum_d<NT>(en, red);
      const double sd = block_sum_d<NT>(ed, red);
      if (tid == 0) a.err_part[(size_t)j * C + c] = make_double2(sn, sd);
    }
    // no peer writes into this CTA after its first transpose in these modes;
    // the cluster leaves together, after every CTA has received its rows
    if (mode == FM_ERR || mode == FM_SIM) {
      asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
      return;
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int s = tid + q * NT;
      const int k1 = s % R1;
      dft<R2, true>(w[q]);
#pragma unroll
      for (int n2 = 1; n2 < R2; ++n2) w[q][n2] = cmul(w[q][n2], cconj(twT[n2 * R1 + k1]));
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int s = tid + q * NT;
      const int k1 = s % R1, rowL = (s / R1) % H, k = s / (R1 * H);
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) Y[rb<F>(k, rowL, k1 * R2 + n2)] = w[q][n2];
    }
  }
  __syncthreads();
  // ---- inverse row stage B: radix R1 -> column x, stored asynchronously
  // into column buffer X of the CTA owning the column
  {
    const int n2 = tid % R2, rowL = (tid / R2) % H, k = tid / (R2 * H);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) v[k1] = Y[rb<F>(k, rowL, k1 * R2 + n2)];
    if (MERGED && !PT_F3_ARRIVE_LATE) asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");  // row data read
    dft<R1, true>(v);
    if (MERGED && PT_F3_ARRIVE_LATE) asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
    if (MERGED) asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");  // peers' too
    const int f = c * H + rowL;
    const uint32_t barX_l = smem_u32(barX);
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      const int x = n1 * R2 + n2;
      const uint32_t rank = (uint32_t)(x / W);
      st_async_f2(mapa_u32(smem_u32(X + cb<F>(k, f, x % W)), rank), v[n1], mapa_u32(barX_l, rank));
    }
  }
  mbar_wait_flag(barX, a.err_flag, a.wait_limit);
  // ---- inverse column stage A: task (k, colL, k1), radix R2 over k2
  {
    float2 w[Q][R2];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int s = tid + q * NT;
      const int colL = s % W, k1 = (s / W) % R1, k = s / (W * R1);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) w[q][k2] = X[cb<F>(k, k1 + R1 * k2, colL)];
      dft<R2, true>(w[q]);
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) w[q][n2] = cmul(w[q][n2], cconj(tw[k1 * R2 + n2]));
    }
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int s = tid + q * NT;
      const int colL = s % W, k1 = (s / W) % R1, k = s / (W * R1);
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) X[cb<F>(k, k1 + R1 * n2, colL)] = w[q][n2];
    }
  }
  __syncthreads();
  // ---- inverse column stage B + epilogue
  {
    const int colL = tid % W, n2 = (tid / W) % R2, k = tid / (W * R2);
    const int col = c * W + colL;
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) v[k1] = X[cb<F>(k, k1 + R1 * n2, colL)];
    dft<R1, true>(v);
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      const int row = n1 * R2 + n2;
      const size_t xi = (((size_t)(j - a.xoff) * K + k) * M + row) * M + col;
      if (mode == FM_CHI || mode == FM_CHIP) {
        // streamed out (evict first: keep L2 for O and P), FP32 or FP16
        if (a.x16) __stcs(reinterpret_cast<unsigned*>(a.X) + xi, half2_bits(v[n1]));
        else __stcs(a.X + xi, v[n1]);
      } else {
        const float2 o = __ldg(a.O + (size_t)(p.x + row) * a.nx + p.y + col);
        const float2 pr = __ldg(Pj + ((size_t)k * M + row) * M + col);
        __stcs(a.X + xi, cadd(cmul(pr, o), v[n1]));
      }
    }
  }
}

}  // namespace ptycho

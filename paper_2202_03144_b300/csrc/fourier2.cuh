// Fused Fourier step, register-resident form (DM, LSQML residual, Fourier
// error, forward simulation).
//
// The K x M x M exit waves of one scan position are split over a cluster of C
// CTAs.  Every 1-D transform of length M = R1 x R2 is done as two register
// radix stages (R1 first, then R2; Cooley-Tukey with the twiddle
// W_M^(n2 k1) between them), so a thread holds R1 complex values at a time
// and shared memory is touched only to exchange data between the stages:
//
//   global -> regs   exit wave z = P_k O_j (DM: 2 phi - psi), thread = one
//                    column slice {rows n1*R2 + n2}
//   column stage 1   radix R1 in registers, twiddle, -> smem   (exchange 1)
//   column stage 2   radix R2 in registers -> pushed to the CTA that owns the
//                    frequency row, through distributed shared memory
//                    (exchange 2 = the column -> row transpose)
//   row stage 1      radix R1, twiddle, -> smem                (exchange 3)
//   row stage 2      radix R2: the thread now holds R2 Fourier pixels of one
//                    row; modulus projection in registers (K = 1) against
//                    sqrt(I) prefetched into shared memory by a bulk async
//                    copy (TMA engine) at kernel start, giving
//                    D = (Pi(Z) - Z) / M^2; first inverse stage (radix R2) in
//                    the same registers, conjugate twiddle  -> smem (4)
//   inverse row B    radix R1 -> pushed back to the column owner (5)
//   inverse col A    radix R2, conjugate twiddle -> smem      (6)
//   inverse col B    radix R1 -> the thread holds spatial rows of one column
//                    -> epilogue straight to global memory.
//
// Six shared-memory round trips per transform pair (two of them across the
// cluster), against twelve for a pass-per-stage shared-memory FFT.  The row
// buffer is laid out (rb()) so that both the stride-R2 reads of row stage 2
// and the unit-stride reads of row stage 1 are free of bank conflicts.
//
// The inverse FFT is unnormalised; 1/M^2 is folded into the projection.  By
// linearity the epilogue needs no second read of psi:
//   LSQML / ePIE: chi = F^-1 D;   DM: psi_new = phi + F^-1 D.
#pragma once
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "common.cuh"
#include "fourier.cuh"

namespace ptycho {

// First-stage radix: 16 for 128 and 256, 8 for 32 and 64, 4 for 16; 24 (= 8 x 3)
// for the mixed-radix sizes 96 (24 x 4) and 192 (24 x 8).
__host__ __device__ constexpr int radix1(int M) {
  return (M % 3 == 0) ? 24 : (M >= 128 ? 16 : (M >= 32 ? 8 : 4));
}

template <int M_, int K_, int C_>
struct F2 {
  static constexpr int M = M_, K = K_, C = C_;
  static constexpr int R1 = radix1(M), R2 = M / R1;
  static constexpr int W = M / C, H = M / C;
  static constexpr int NT = K * W * R2;       // threads (= stage-1 tasks of either axis)
  static constexpr int Q = R1 / R2;           // stage-2 tasks per thread
  static constexpr int L = K * M * W;         // complex elements per CTA
  static constexpr int PB = M + (R2 >= 16 ? 0 : (R2 == 8 ? 8 : 4));  // row pitch
  static constexpr int SBUF = (K * H * PB > L) ? K * H * PB : L;
  static constexpr int NRED = 64;
  static_assert(R1 * R2 == M && R1 % R2 == 0 && R1 <= 24, "radix split");
  static_assert(M % C == 0 && W >= 1, "cluster split");
  static_assert(NT % 32 == 0 && NT <= 1024, "threads");
};

// bytes of dynamic shared memory: data, twiddle table, amplitude tile,
// reduction scratch, mbarrier
template <class F>
__host__ __device__ constexpr size_t fourier2_smem() {
  return (size_t)F::SBUF * 8 + (size_t)F::M * 16 + (size_t)F::H * F::M * 4 + F::NRED * 8 + 16;
}

// Row-buffer index of column x: XOR swizzle inside groups of 16 (an explicit
// pad element after every 16 columns measured 6% slower at M = 256).
template <class F>
__device__ __forceinline__ int rb(int k, int rowL, int x) {
  const int sx = x ^ ((x >> 4) & (F::R2 - 1));
  return (k * F::H + rowL) * F::PB + sx;
}
template <class F>
__device__ __forceinline__ int cb(int k, int r, int colL) {
  return (k * F::M + r) * F::W + colL;
}

// --- cluster barriers ----------------------------------------------------
// Read-after-write: release the shared-memory writes, acquire the peers'.
__device__ __forceinline__ void cluster_sync_rw() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Write-after-read: every CTA has consumed (into registers) what it read.
__device__ __forceinline__ void cluster_sync_war() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\tbarrier.cluster.wait.aligned;" ::: "memory");
}

// Shared::cluster address of the same offset in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t mapa_u32(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster_f2(uint32_t addr, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(v.x), "f"(v.y) : "memory");
}

// --- bulk async copy (TMA engine) of the amplitude tile -------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Bounded wait on phase 0 of the barrier; returns false (and the caller flags
// an error) if the copy has not landed after ~2^22 polls.
__device__ __forceinline__ bool mbar_wait0(uint64_t* bar) {
  uint32_t done = 0;
  for (int i = 0; i < (1 << 22) && !done; ++i) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar))
        : "memory");
  }
  return done != 0;
}

struct Fourier2Args {
  const float2* O;
  int nx;
  const float2* P;        // probe [K][M][M], or the shifted table [bins][K][M][M]
  const unsigned short* pbin;  // sub-pixel bin of each position, or NULL
  const int2* pos;
  float2* X;
  const void* amp;
  const float* amp_scale;
  int istore;
  float* I_out;
  double2* err_part;
  const float2* tw2;      // tw2[k1 * R2 + n2] = exp(-2 pi i n2 k1 / M)
  int* err_flag;          // set to 1 if a bounded wait gave up
  int wait_limit;         // polls of a cluster-transpose wait before it gives up
  int x16;                // residual passes: X holds chi as FP16 complex (__half2)
  int j0;                 // first position of the launch
  int nj;                 // positions of the launch (persistent kernels walk them)
  int xoff;               // X holds positions from xoff on (position-blocked residuals)
  int mode;
};

// A complex value rounded to FP16, as the 32-bit pattern of a __half2.
__device__ __forceinline__ unsigned half2_bits(float2 v) {
  const __half2 h = __float22half2_rn(v);
  return *reinterpret_cast<const unsigned*>(&h);
}

// Detector-plane factor f with D = f Psi (before the 1/M^2 of the inverse
// transform), from the stored amplitude am = sqrt(I) (< 0: masked) and
// A^2 = sum_k |Psi_k|^2:
//   amplitude likelihood  f = sqrt(I)/A - 1  (projection minus identity;
//                         A^2 <= 1e-38 counts as zero modulus: f = -1)
//   Poisson likelihood    f = (I - A^2) / (I + A^2)  (FM_CHIP: one Newton
//                         step of the pixel's negative log-likelihood along
//                         its gradient; 0 where I + A^2 = 0)
// masked pixels f = 0.
__device__ __forceinline__ float proj_factor(int mode, float am, float A2) {
  if (am < 0.f) return 0.f;
  if (mode == FM_CHIP) {
    const float I = am * am, d = I + A2;
    return d > 0.f ? __fdividef(I - A2, d) : 0.f;
  }
  return (A2 > 1e-38f ? am * rsqrtf(A2) : 0.f) - 1.f;
}

// IST >= 0: storage format fixed at compile time (0 f32, 1 f16, 2 bf16);
// -1: read from the arguments.
template <int IST>
__device__ __forceinline__ float amp_at(const Fourier2Args& a, const void* amp_s, int idx, float scale) {
  const int ist = IST >= 0 ? IST : a.istore;
  if (ist == 0) return reinterpret_cast<const float*>(amp_s)[idx];
  if (ist == 1) return __half2float(reinterpret_cast<const __half*>(amp_s)[idx]) * scale;
  return __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(amp_s)[idx]) * scale;
}

// MODE_T / IST_T >= 0 compile one mode / amplitude format (the hot LSQML and
// DM passes); -1 takes them from the arguments.
template <int M, int K, int C, int MODE_T = -1, int IST_T = -1>
__global__ void __launch_bounds__(F2<M, K, C>::NT, (F2<M, K, C>::R1 > 16 ? 1 : (F2<M, K, C>::NT <= 256 ? 4 : (F2<M, K, C>::NT <= 512 ? 2 : 1)))) k_fourier2(Fourier2Args a) {
  using F = F2<M, K, C>;
  constexpr int R1 = F::R1, R2 = F::R2, W = F::W, H = F::H, NT = F::NT, Q = F::Q;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* buf = reinterpret_cast<float2*>(smem_raw);
  float2* tw = buf + F::SBUF;   // tw[k1 * R2 + n2] = W_M^(n2 k1)
  float2* twT = tw + M;          // twT[n2 * R1 + k1], the same values transposed
  unsigned char* amp_s = reinterpret_cast<unsigned char*>(twT + M);
  double* red = reinterpret_cast<double*>(amp_s + (size_t)H * M * 4);
  uint64_t* bar = reinterpret_cast<uint64_t*>(red + F::NRED);

  pdl_wait();
  pdl_launch();
  const int tid = threadIdx.x;
  const int c = (C > 1) ? (int)(blockIdx.x % C) : 0;
  const int j = a.j0 + (int)(blockIdx.x / C);
  // probe of this position (sub-pixel: its bin of the shifted-probe table)
  const float2* Pj = a.pbin ? a.P + (size_t)__ldg(a.pbin + j) * (K * M * M) : a.P;
  const int mode = MODE_T >= 0 ? MODE_T : a.mode;
  const int istore = IST_T >= 0 ? IST_T : a.istore;
  const int2 p = a.pos[j];
  const bool need_amp = mode != FM_SIM;

  // prefetch this CTA's rows of sqrt(I) (contiguous in global memory)
  if (tid == 0) {
    mbar_init(bar, 1);
    if (need_amp) {
      const size_t esz = istore == 0 ? 4 : 2;
      const unsigned char* src = reinterpret_cast<const unsigned char*>(a.amp) + ((size_t)j * M + c * H) * M * esz;
      bulk_load(amp_s, src, (uint32_t)(H * M * esz), bar);
    }
  }
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
    // probe values first, then the object in groups of four: bounds the number
    // of loads in flight per thread (and so the registers they occupy)
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) v[n1] = __ldg(Pj + ((size_t)k * M + n1 * R2 + n2) * M + col);
    const float2* orow = a.O + (size_t)(p.x + n2) * a.nx + p.y + col;
#pragma unroll
    for (int g0 = 0; g0 < R1; g0 += 4) {
      float2 o[4];
#pragma unroll
      for (int i = 0; i < 4 && g0 + i < R1; ++i) o[i] = __ldg(orow + (size_t)(g0 + i) * R2 * a.nx);
#pragma unroll
      for (int i = 0; i < 4 && g0 + i < R1; ++i) v[g0 + i] = cmul(v[g0 + i], o[i]);
      asm volatile("" ::: "memory");
    }
    if (mode == FM_DM) {
      const float2* xrow = a.X + (((size_t)(j - a.xoff) * K + k) * M + n2) * M + col;
#pragma unroll
      for (int n1 = 0; n1 < R1; ++n1) v[n1] = csub(cscale(v[n1], 2.f), xrow[(size_t)n1 * R2 * M]);
    }
    __syncthreads();  // twiddle table and mbarrier initialisation
    dft<R1, false>(v);
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) v[k1] = cmul(v[k1], tw[k1 * R2 + n2]);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) buf[cb<F>(k, k1 * R2 + n2, colL)] = v[k1];
  }
  __syncthreads();
  // ---- column stage 2: task (k, colL, k1) -> frequency rows k1 + R1*k2
  {
    float2 w[Q][R2];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int s = tid + q * NT;
      const int colL = s % W, k1 = (s / W) % R1, k = s / (W * R1);
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) w[q][n2] = buf[cb<F>(k, k1 * R2 + n2, colL)];
      dft<R2, false>(w[q]);
    }
    // transpose: frequency row f goes to CTA f / H, row f % H of its row buffer
    if constexpr (C > 1) cluster_sync_war();
    else __syncthreads();
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int s = tid + q * NT;
      const int colL = s % W, k1 = (s / W) % R1, k = s / (W * R1);
      const int col = c * W + colL;
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) {
        const int f = k1 + R1 * k2;
        if constexpr (C > 1) {
          st_cluster_f2(mapa_u32(smem_u32(buf + rb<F>(k, f % H, col)), (uint32_t)(f / H)), w[q][k2]);
        } else {
          buf[rb<F>(k, f % H, col)] = w[q][k2];
        }
      }
    }
    if constexpr (C > 1) cluster_sync_rw();
    else __syncthreads();
  }
  // ---- row stage 1: task (k, rowL, n2'), columns n1'*R2 + n2'
  {
    const int n2 = tid % R2, rowL = (tid / R2) % H, k = tid / (R2 * H);
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) v[n1] = buf[rb<F>(k, rowL, n1 * R2 + n2)];
    dft<R1, false>(v);
#pragma unroll
    for (int k1 = 1; k1 < R1; ++k1) v[k1] = cmul(v[k1], tw[k1 * R2 + n2]);
    // each thread writes back exactly the slots {i*R2 + n2} it read: no
    // write-after-read barrier needed
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) buf[rb<F>(k, rowL, k1 * R2 + n2)] = v[k1];
  }
  __syncthreads();
  // ---- row stage 2 (+ projection + first inverse stage)
  float scale = 1.f;
  if (need_amp && istore != 0) scale = __ldg(a.amp_scale + j);
  if (need_amp) {
    // every thread waits on the barrier (the copy's writes become visible)
    if (!mbar_wait0(bar)) atomicExch(a.err_flag, 1);
  }
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
      for (int n2 = 0; n2 < R2; ++n2) w[q][n2] = buf[rb<F>(k, rowL, k1 * R2 + n2)];
      dft<R2, false>(w[q]);
      if constexpr (K == 1) {
        const int ky = c * H + rowL;
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) {
          const int kx = k1 + R1 * k2;
          const float A2 = cabs2(w[q][k2]);
          if (mode == FM_SIM) {
            a.I_out[((size_t)j * M + ((ky + M / 2) % M)) * M + ((kx + M / 2) % M)] = A2;
          } else {
            const float am = amp_at<IST_T>(a, amp_s, rowL * M + kx, scale);
            if (mode == FM_ERR) {
              if (am >= 0.f) {
                const float d = sqrtf(A2) - am;
                en = fmaf(d, d, en);
                ed = fmaf(am, am, ed);
              }
            } else {
              const float fct = proj_factor(mode, am, A2);
              w[q][k2] = cscale(w[q][k2], fct * inv);
            }
          }
        }
      }
    }
    if constexpr (K > 1) {
      // modes live in different threads: project through shared memory
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int s = tid + q * NT;
        const int k1 = s % R1, rowL = (s / R1) % H, k = s / (R1 * H);
#pragma unroll
        for (int k2 = 0; k2 < R2; ++k2) buf[rb<F>(k, rowL, k1 * R2 + k2)] = w[q][k2];
      }
      __syncthreads();
      for (int px = tid; px < H * M; px += NT) {
        const int rowL = px / M, pp = px % M;  // pp = k1 * R2 + k2 storage slot
        const int kx = pp / R2 + R1 * (pp % R2);
        const int ky = c * H + rowL;
        float2 z[K];
        float A2 = 0.f;
#pragma unroll
        for (int k = 0; k < K; ++k) {
          z[k] = buf[rb<F>(k, rowL, pp)];
          A2 += cabs2(z[k]);
        }
        if (mode == FM_SIM) {
          a.I_out[((size_t)j * M + ((ky + M / 2) % M)) * M + ((kx + M / 2) % M)] = A2;
          continue;
        }
        const float am = amp_at<IST_T>(a, amp_s, rowL * M + kx, scale);
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
        for (int k = 0; k < K; ++k) buf[rb<F>(k, rowL, pp)] = cscale(z[k], fct * inv);
      }
      __syncthreads();
      if (mode == FM_DM || mode == FM_CHI || mode == FM_CHIP) {
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          const int s = tid + q * NT;
          const int k1 = s % R1, rowL = (s / R1) % H, k = s / (R1 * H);
#pragma unroll
          for (int k2 = 0; k2 < R2; ++k2) w[q][k2] = buf[rb<F>(k, rowL, k1 * R2 + k2)];
        }
      }
    }
    if (mode == FM_ERR) {
      const double sn = block_sum_d<NT>(en, red);
      const double sd = block_sum_d<NT>(ed, red);
      if (tid == 0) a.err_part[(size_t)j * C + c] = make_double2(sn, sd);
    }
    if (mode == FM_ERR || mode == FM_SIM) return;  // no DSMEM access after the transpose
    // inverse row stage A: radix R2 over k2', conjugate twiddle (threads of a
    // warp differ in k1, so read the transposed table: no bank conflicts)
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int s = tid + q * NT;
      const int k1 = s % R1;
      dft<R2, true>(w[q]);
#pragma unroll
      for (int n2 = 1; n2 < R2; ++n2) w[q][n2] = cmul(w[q][n2], cconj(twT[n2 * R1 + k1]));
    }
    // written back to the slots {k1*R2 + i} this thread read in row stage 2
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int s = tid + q * NT;
      const int k1 = s % R1, rowL = (s / R1) % H, k = s / (R1 * H);
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) buf[rb<F>(k, rowL, k1 * R2 + n2)] = w[q][n2];
    }
  }
  __syncthreads();
  // ---- inverse row stage B: task (k, rowL, n2'), radix R1 -> columns n1'*R2 + n2'
  {
    const int n2 = tid % R2, rowL = (tid / R2) % H, k = tid / (R2 * H);
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) v[k1] = buf[rb<F>(k, rowL, k1 * R2 + n2)];
    dft<R1, true>(v);
    // transpose back: column x goes to CTA x / W, row c*H + rowL of its column buffer
    if constexpr (C > 1) cluster_sync_war();
    else __syncthreads();
    const int f = c * H + rowL;
#pragma unroll
    for (int n1 = 0; n1 < R1; ++n1) {
      const int x = n1 * R2 + n2;
      if constexpr (C > 1) {
        st_cluster_f2(mapa_u32(smem_u32(buf + cb<F>(k, f, x % W)), (uint32_t)(x / W)), v[n1]);
      } else {
        buf[cb<F>(k, f, x % W)] = v[n1];
      }
    }
    if constexpr (C > 1) cluster_sync_rw();
    else __syncthreads();
  }
  // ---- inverse column stage A: task (k, colL, k1), radix R2 over k2
  {
    float2 w[Q][R2];
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int s = tid + q * NT;
      const int colL = s % W, k1 = (s / W) % R1, k = s / (W * R1);
#pragma unroll
      for (int k2 = 0; k2 < R2; ++k2) w[q][k2] = buf[cb<F>(k, k1 + R1 * k2, colL)];
      dft<R2, true>(w[q]);
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) w[q][n2] = cmul(w[q][n2], cconj(tw[k1 * R2 + n2]));
    }
    // value (k1, n2) goes to row k1 + R1*n2: the same rows this task read, so
    // no write-after-read barrier is needed
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int s = tid + q * NT;
      const int colL = s % W, k1 = (s / W) % R1, k = s / (W * R1);
#pragma unroll
      for (int n2 = 0; n2 < R2; ++n2) buf[cb<F>(k, k1 + R1 * n2, colL)] = w[q][n2];
    }
  }
  __syncthreads();
  // ---- inverse column stage B + epilogue: thread = (k, colL, n2), rows n1*R2 + n2
  {
    const int colL = tid % W, n2 = (tid / W) % R2, k = tid / (W * R2);
    const int col = c * W + colL;
#pragma unroll
    for (int k1 = 0; k1 < R1; ++k1) v[k1] = buf[cb<F>(k, k1 + R1 * n2, colL)];
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

// Learned warm start: a convolutional encoder-decoder that maps one
// diffraction frame, log(1 + I) of a 128 x 128 detector-centred pattern, to
// the amplitude and phase of the central 64 x 64 object patch under the
// probe.  Predicted patches are stitched into the initial object of a DM or
// LSQML reconstruction (the iterations have the last word).
//
// Layers (3 x 3 kernels, padding 1; "s2" = stride 2, "up" = nearest x2
// upsampling of the input folded into the convolution's index map):
//   128^2:  1 ->  16            relu
//    64^2: 16 ->  32  s2        relu
//    32^2: 32 ->  64  s2        relu
//    16^2: 64 -> 128  s2        relu
//     8^2: 128 -> 256 s2        relu
//     4^2: 256 -> 256 s2, 256 -> 256   relu
//     8^2: 256 -> 128 up        relu
//    16^2: 128 -> 64  up        relu
//    32^2: 64 ->  32  up        relu
//    64^2: 32 ->  16  up        relu, then 16 -> 2 (amplitude, phase)
// 1,964,690 parameters (1,963,440 weights, 1,250 biases).  Weights and activations are stored in BF16, all
// sums are FP32 (the last layer's output and every gradient are FP32).  Each
// reduction (weight and bias gradients, loss) runs in a fixed order, so a
// training step is deterministic.
#pragma once
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc.cuh"

namespace ptycho {

constexpr int NET_IN = 128, NET_OUT = 64, NET_LAYERS = 12;

struct NetLayer {
  int ci, co, hin, win, hout, wout, stride, up, relu;
};

__host__ __device__ constexpr NetLayer net_layer(int l) {
  return l == 0    ? NetLayer{1, 16, 128, 128, 128, 128, 1, 0, 1}
         : l == 1  ? NetLayer{16, 32, 128, 128, 64, 64, 2, 0, 1}
         : l == 2  ? NetLayer{32, 64, 64, 64, 32, 32, 2, 0, 1}
         : l == 3  ? NetLayer{64, 128, 32, 32, 16, 16, 2, 0, 1}
         : l == 4  ? NetLayer{128, 256, 16, 16, 8, 8, 2, 0, 1}
         : l == 5  ? NetLayer{256, 256, 8, 8, 4, 4, 2, 0, 1}
         : l == 6  ? NetLayer{256, 256, 4, 4, 4, 4, 1, 0, 1}
         : l == 7  ? NetLayer{256, 128, 4, 4, 8, 8, 1, 1, 1}
         : l == 8  ? NetLayer{128, 64, 8, 8, 16, 16, 1, 1, 1}
         : l == 9  ? NetLayer{64, 32, 16, 16, 32, 32, 1, 1, 1}
         : l == 10 ? NetLayer{32, 16, 32, 32, 64, 64, 1, 1, 1}
                   : NetLayer{16, 2, 64, 64, 64, 64, 1, 0, 0};
}

// Input coordinate of output coordinate o and tap d (0..2) of a layer, or -1
// outside the (virtual, upsampled) input.
__device__ __forceinline__ int net_src(int o, int d, int stride, int up, int hin) {
  const int v = stride * o + d - 1;
  const int hv = up ? 2 * hin : hin;
  if (v < 0 || v >= hv) return -1;
  return up ? (v >> 1) : v;
}

// activation storage: BF16 (the method) or FP32 (verification mode)
__device__ __forceinline__ float ldact(const __nv_bfloat16* p, size_t i) { return __bfloat162float(p[i]); }
__device__ __forceinline__ float ldact(const float* p, size_t i) { return p[i]; }
__device__ __forceinline__ void stact(__nv_bfloat16* p, size_t i, float v) { p[i] = __float2bfloat16_rn(v); }
__device__ __forceinline__ void stact(float* p, size_t i, float v) { p[i] = v; }

struct ConvArgs {
  const void* in;            // [B][ci][hin][win] activations (TA)
  const __nv_bfloat16* w;    // [co][ci][9]
  const float* b;            // [co]
  void* out;                 // [B][co][hout][wout], bf16 (or f32 for the last layer)
  const float* dout;         // backward: delta of this layer [B][co][hout][wout]
  float* din;                // backward data: delta of the previous layer
  const void* mask;          // backward data: previous layer's output (relu mask, TA) or NULL
  float* wpart;              // backward weights: partials [chunks][co][ci][9]
  int B, ci, co, hin, win, hout, wout, stride, up, relu;
};

constexpr int CV_NT = 256, CV_CO = 16, CV_CI = 16;

// Forward: thread = one output pixel, CV_CO output channels.
template <typename TA, bool OUT_F32>
__global__ void __launch_bounds__(CV_NT) k_conv_fwd(ConvArgs a) {
  const TA* in = reinterpret_cast<const TA*>(a.in);
  __shared__ __align__(16) float ws[CV_CI][9][CV_CO];
  const int tid = threadIdx.x;
  const long long npix = (long long)a.B * a.hout * a.wout;
  const long long p = (long long)blockIdx.x * CV_NT + tid;
  const bool valid = p < npix;
  const int n = valid ? (int)(p / (a.hout * a.wout)) : 0;
  const int y = valid ? (int)((p / a.wout) % a.hout) : 0;
  const int x = valid ? (int)(p % a.wout) : 0;
  const int co0 = blockIdx.y * CV_CO;
  float acc[CV_CO];
#pragma unroll
  for (int c = 0; c < CV_CO; ++c) acc[c] = (co0 + c < a.co) ? a.b[co0 + c] : 0.f;
  int sy[3], sx[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    sy[d] = net_src(y, d, a.stride, a.up, a.hin);
    sx[d] = net_src(x, d, a.stride, a.up, a.win);
  }
  for (int ci0 = 0; ci0 < a.ci; ci0 += CV_CI) {
    __syncthreads();
    for (int i = tid; i < CV_CI * 9 * CV_CO; i += CV_NT) {
      const int ci = i / (9 * CV_CO), t = (i / CV_CO) % 9, c = i % CV_CO;
      ws[ci][t][c] = (ci0 + ci < a.ci && co0 + c < a.co)
                         ? __bfloat162float(a.w[((size_t)(co0 + c) * a.ci + ci0 + ci) * 9 + t])
                         : 0.f;
    }
    __syncthreads();
    if (valid) {
      const int nci = min(CV_CI, a.ci - ci0);
      for (int ci = 0; ci < nci; ++ci) {
        const TA* src = in + ((size_t)n * a.ci + ci0 + ci) * a.hin * a.win;
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
          if (sy[dy] < 0) continue;
#pragma unroll
          for (int dx = 0; dx < 3; ++dx) {
            if (sx[dx] < 0) continue;
            const float v = ldact(src, (size_t)sy[dy] * a.win + sx[dx]);
            const float4* wv = reinterpret_cast<const float4*>(&ws[ci][dy * 3 + dx][0]);
#pragma unroll
            for (int q = 0; q < CV_CO / 4; ++q) {
              const float4 w4 = wv[q];
              acc[4 * q + 0] = fmaf(w4.x, v, acc[4 * q + 0]);
              acc[4 * q + 1] = fmaf(w4.y, v, acc[4 * q + 1]);
              acc[4 * q + 2] = fmaf(w4.z, v, acc[4 * q + 2]);
              acc[4 * q + 3] = fmaf(w4.w, v, acc[4 * q + 3]);
            }
          }
        }
      }
    }
  }
  if (!valid) return;
#pragma unroll
  for (int c = 0; c < CV_CO; ++c) {
    if (co0 + c >= a.co) continue;
    float r = acc[c];
    if (a.relu) r = fmaxf(r, 0.f);
    const size_t o = (((size_t)n * a.co + co0 + c) * a.hout + y) * a.wout + x;
    if (OUT_F32) reinterpret_cast<float*>(a.out)[o] = r;
    else stact(reinterpret_cast<TA*>(a.out), o, r);
  }
}

// Forward on the tensor cores (implicit GEMM): D[pixel][co] =
// sum_k A[pixel][k] B[co][k] with k = ci * 9 + tap, A gathered from the
// BF16 activations (im2col, zero outside the input), B = the BF16 weights.
// CTA = 128 output pixels x all output channels (NP = co rounded up to 16)
// x one slice of the K chunks (split-K for the deep layers, whose few pixels
// would otherwise leave most SMs idle).  Two shared-memory stages: the 128
// threads gather chunk c+1 into one stage while the tensor cores run the four
// K=16 MMAs of chunk c from the other; each stage's mbarrier phase tells when
// its MMAs are done.  The FP32 accumulator lives in tensor memory.
// Epilogue: tensor memory -> registers -> bias, ReLU, BF16 store (ksplit = 1)
// or an FP32 partial tile (ksplit > 1, summed in order by k_conv_tc_reduce).
constexpr int TC_KC = 64;
template <int NP>
__host__ __device__ constexpr int tc_ncols() { return NP < 32 ? 32 : NP; }
template <int NP>
__host__ __device__ constexpr size_t conv_tc_smem() {
  // two (A, B) stages, the per-pixel tap offsets [9][128], mbarriers
  return 2 * ((size_t)128 * TC_KC * 2 + (size_t)NP * TC_KC * 2) + 9 * 128 * 4 + 64;
}

// NHWC = true (inference): activations channel-last [B][h][w][c] and the
// weights tap-major [co][tap][ci], i.e. k = tap * ci + c.  With ci a power of
// two >= 8, each group of 8 consecutive k is 8 channels of one tap of one
// input pixel: one 16-byte load instead of eight gathered elements; the
// output tile is written as 16-byte channel vectors (the last layer stays
// FP32 [B][co][h][w]).
template <bool OUT_F32, int NP, bool NHWC = false>
__global__ void __launch_bounds__(128) k_conv_fwd_tc(ConvArgs a, int ksplit, float* part, int* err_flag) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  constexpr size_t ABYTES = 128 * TC_KC * 2, BBYTES = (size_t)NP * TC_KC * 2;
  unsigned char* stage[2] = {smem_raw, smem_raw + ABYTES + BBYTES};
  int* offs = reinterpret_cast<int*>(smem_raw + 2 * (ABYTES + BBYTES));  // [9][128]
  uint64_t* bar = reinterpret_cast<uint64_t*>(offs + 9 * 128);            // [2]
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  constexpr uint32_t LBO = 128, SBO = (TC_KC / 8) * 128;
  constexpr uint32_t NCOLS = tc_ncols<NP>();
  const __nv_bfloat16* in = reinterpret_cast<const __nv_bfloat16*>(a.in);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int npix = a.B * a.hout * a.wout;  // < 2^31 for every supported batch
  const int p = blockIdx.x * 128 + tid;
  const bool valid = p < npix;
  const int hw = a.hout * a.wout;
  const int n = valid ? p / hw : 0;
  const int yx = valid ? p - n * hw : 0;
  const int y = yx / a.wout, x = yx - y * a.wout;
  // input offset of each tap within a channel plane (-1 outside), kept in
  // shared memory so that the gather indexes it by the tap of each k
#pragma unroll
  for (int t = 0; t < 9; ++t) {
    const int yy = net_src(y, t / 3, a.stride, a.up, a.hin), xx = net_src(x, t % 3, a.stride, a.up, a.win);
    offs[t * 128 + tid] = (valid && yy >= 0 && xx >= 0) ? yy * a.win + xx : -1;
  }
  if (tid == 0) {
    tc::mbar_init1(&bar[0]);
    tc::mbar_init1(&bar[1]);
  }
  if (warp == 0) tc::tmem_alloc(tslot, NCOLS);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *tslot;
  const int K = a.ci * 9;
  const int nchunk = (K + TC_KC - 1) / TC_KC;
  const int c_begin = (int)(((long long)nchunk * blockIdx.y) / ksplit);
  const int c_end = (int)(((long long)nchunk * (blockIdx.y + 1)) / ksplit);
  const size_t plane = (size_t)a.hin * a.win;
  const __nv_bfloat16* src = in + (size_t)n * a.ci * plane;
  const bool wvec = (K % 8) == 0;
  constexpr uint32_t idesc = tc::idesc_bf16_f32(128, NP);
  uint32_t ph[2] = {0u, 0u};
  bool pending[2] = {false, false};  // a commit on this stage not yet waited for
  bool ok = true;
  for (int c = c_begin; c < c_end; ++c) {
    const int s = (c - c_begin) & 1;
    if (pending[s]) {  // the MMAs that read this stage two chunks ago must be done
      if (!tc::mbar_wait(&bar[s], ph[s])) ok = false;
      ph[s] ^= 1u;
      pending[s] = false;
      tc::fence_after();
    }
    unsigned char* As = stage[s];
    unsigned char* Bs = stage[s] + ABYTES;
    const int k0 = c * TC_KC;
    if (NHWC && a.ci >= 8) {
      // A: 8 groups of 8 channels of one tap, 16-byte loads all in flight
      const int lg = 31 - __clz(a.ci);
      const __nv_bfloat16* img = in + (size_t)n * plane * a.ci;
      uint4 q[TC_KC / 8];
#pragma unroll
      for (int g = 0; g < TC_KC / 8; ++g) {
        const int k = k0 + 8 * g;
        const int o = k < K ? offs[(k >> lg) * 128 + tid] : -1;
        q[g] = o >= 0 ? __ldg(reinterpret_cast<const uint4*>(img + (size_t)o * a.ci + (k & (a.ci - 1))))
                      : make_uint4(0u, 0u, 0u, 0u);
      }
#pragma unroll
      for (int g = 0; g < TC_KC / 8; ++g)
        *reinterpret_cast<uint4*>(As + (tid >> 3) * SBO + g * LBO + (tid & 7) * 16) = q[g];
    } else if (a.ci >= 8) {
      // NCHW with tap-major weights: k = tap * ci + c, so a group of eight k
      // is one tap (one offset) and eight channel planes
      const int lg = 31 - __clz(a.ci);
      const unsigned short* src16 = reinterpret_cast<const unsigned short*>(src);
      uint32_t w[TC_KC / 2];
#pragma unroll
      for (int g = 0; g < TC_KC / 8; ++g) {
        const int k = k0 + 8 * g;
        const int o = k < K ? offs[(k >> lg) * 128 + tid] : -1;
        const unsigned short* pc = src16 + (size_t)(k & (a.ci - 1)) * plane + (o >= 0 ? o : 0);
        unsigned short raw[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) raw[e] = o >= 0 ? __ldg(pc + (size_t)e * plane) : (unsigned short)0;
#pragma unroll
        for (int e = 0; e < 4; ++e) w[4 * g + e] = (uint32_t)raw[2 * e] | ((uint32_t)raw[2 * e + 1] << 16);
      }
#pragma unroll
      for (int g = 0; g < TC_KC / 8; ++g)
        *reinterpret_cast<uint4*>(As + (tid >> 3) * SBO + g * LBO + (tid & 7) * 16) =
            make_uint4(w[4 * g], w[4 * g + 1], w[4 * g + 2], w[4 * g + 3]);
    } else {
    // A: this thread's pixel (row tid), 64 values of k = ci * 9 + tap, in
    // two halves of 32 independent loads (one memory latency per half, not
    // one per group of 8); halves past the end of K are zeros (NHWC with
    // ci = 1 is the same layout)
    int ci = k0 / 9, t = k0 - 9 * (k0 / 9);
    const unsigned short* src16 = reinterpret_cast<const unsigned short*>(src);
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      uint32_t w[16];
      if (k0 + 32 * hh < K) {
        unsigned short raw[32];
#pragma unroll
        for (int e = 0; e < 32; ++e) {
          const int o = ci < a.ci ? offs[t * 128 + tid] : -1;
          raw[e] = o >= 0 ? __ldg(src16 + ci * plane + o) : (unsigned short)0;
          if (++t == 9) {
            t = 0;
            ++ci;
          }
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) w[e] = (uint32_t)raw[2 * e] | ((uint32_t)raw[2 * e + 1] << 16);
      } else {
#pragma unroll
        for (int e = 0; e < 16; ++e) w[e] = 0u;
      }
#pragma unroll
      for (int g = 0; g < 4; ++g)
        *reinterpret_cast<uint4*>(As + (tid >> 3) * SBO + (4 * hh + g) * LBO + (tid & 7) * 16) =
            make_uint4(w[4 * g], w[4 * g + 1], w[4 * g + 2], w[4 * g + 3]);
    }
    }
    // B: weight rows (output channels) tid, tid + 128
    for (int r = tid; r < NP; r += 128) {
#pragma unroll
      for (int g = 0; g < TC_KC / 8; ++g) {
        const int kb = k0 + g * 8;
        uint4 q;
        if (wvec && r < a.co && kb + 8 <= K) {
          q = __ldg(reinterpret_cast<const uint4*>(a.w + (size_t)r * K + kb));
        } else {
          __align__(16) __nv_bfloat16 v8[8];
#pragma unroll
          for (int e = 0; e < 8; ++e)
            v8[e] = (r < a.co && kb + e < K) ? a.w[(size_t)r * K + kb + e] : __float2bfloat16_rn(0.f);
          q = *reinterpret_cast<const uint4*>(v8);
        }
        *reinterpret_cast<uint4*>(Bs + (r >> 3) * SBO + g * LBO + (r & 7) * 16) = q;
      }
    }
    // generic-proxy writes -> visible to the tensor cores' async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
#pragma unroll
      for (int kk = 0; kk < TC_KC / 16; ++kk) {
        const uint64_t ad = tc::smem_desc(As + kk * 2 * LBO, LBO, SBO);
        const uint64_t bd = tc::smem_desc(Bs + kk * 2 * LBO, LBO, SBO);
        tc::mma_bf16(tbase, ad, bd, idesc, (c > c_begin || kk > 0) ? 1u : 0u);
      }
      tc::commit(&bar[s]);
    }
    pending[s] = true;
  }
  // drain the stages still in flight
  const int nloc = c_end - c_begin;
#pragma unroll
  for (int s = 0; s < 2; ++s)
    if (pending[s] && !tc::mbar_wait(&bar[s], ph[s])) ok = false;
  tc::fence_after();
  if (!ok && tid == 0) atomicExch(err_flag, 1);
  // epilogue: this warp's 32 lanes = pixels blockIdx.x*128 + 32*warp + lane
#pragma unroll 1
  for (int c0 = 0; c0 < NP; c0 += 16) {
    float v[16];
    tc::tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
    if (NHWC && !OUT_F32 && ksplit == 1 && valid) {
      // 16 channels of this pixel: two 16-byte stores (co is a multiple of 16)
      uint32_t pk[8];
#pragma unroll
      for (int j = 0; j < 16; j += 2) {
        float r0 = v[j] + a.b[c0 + j], r1 = v[j + 1] + a.b[c0 + j + 1];
        if (a.relu) r0 = fmaxf(r0, 0.f), r1 = fmaxf(r1, 0.f);
        const __nv_bfloat162 h2 = __floats2bfloat162_rn(r0, r1);
        pk[j / 2] = *reinterpret_cast<const uint32_t*>(&h2);
      }
      uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(a.out) + (size_t)p * a.co + c0);
      dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
    } else if (valid) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int co = c0 + j;
        if (co >= a.co) continue;
        if (ksplit > 1) {
          part[((size_t)blockIdx.y * a.co + co) * npix + p] = nloc > 0 ? v[j] : 0.f;
          continue;
        }
        float r = v[j] + a.b[co];
        if (a.relu) r = fmaxf(r, 0.f);
        const size_t o = (((size_t)n * a.co + co) * a.hout + y) * a.wout + x;
        if (OUT_F32) reinterpret_cast<float*>(a.out)[o] = r;
        else reinterpret_cast<__nv_bfloat16*>(a.out)[o] = __float2bfloat16_rn(r);
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tbase, NCOLS);
}

// Split-K epilogue: out = act(bias + sum of the ksplit partial tiles, in
// order), into [B][co][h][w] or (NHWC, BF16) [B][h][w][co].
template <bool OUT_F32, bool NHWC = false>
__global__ void k_conv_tc_reduce(ConvArgs a, int ksplit, const float* __restrict__ part) {
  const long long npix = (long long)a.B * a.hout * a.wout;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npix * a.co;
       i += (long long)gridDim.x * blockDim.x) {
    const int co = (int)(i / npix);
    const long long p = i % npix;
    float r = a.b[co];
    for (int s = 0; s < ksplit; ++s) r += part[((size_t)s * a.co + co) * npix + p];
    if (a.relu) r = fmaxf(r, 0.f);
    const int n = (int)(p / (a.hout * a.wout));
    const int yx = (int)(p % (a.hout * a.wout));
    const size_t o = (NHWC && !OUT_F32) ? (size_t)p * a.co + co : ((size_t)n * a.co + co) * a.hout * a.wout + yx;
    if (OUT_F32) reinterpret_cast<float*>(a.out)[o] = r;
    else reinterpret_cast<__nv_bfloat16*>(a.out)[o] = __float2bfloat16_rn(r);
  }
}

// First layer of the inference forward (1 -> 16 channels, 3 x 3, stride 1)
// on the CUDA cores: 144 FMAs per pixel do not pay for a tensor-core tile.
// Thread = one output pixel; output channel-last BF16 (two 16-byte stores).
__global__ void __launch_bounds__(256) k_conv_first_nhwc(ConvArgs a) {
  __shared__ float ws[16][9];
  __shared__ float bs[16];
  for (int i = threadIdx.x; i < 16 * 9; i += blockDim.x) ws[i / 9][i % 9] = __bfloat162float(a.w[i]);
  if (threadIdx.x < 16) bs[threadIdx.x] = a.b[threadIdx.x];
  __syncthreads();
  const __nv_bfloat16* in = reinterpret_cast<const __nv_bfloat16*>(a.in);
  const int hw = a.hout * a.wout, npix = a.B * hw;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
    const int n = p / hw, yx = p - n * hw, y = yx / a.wout, x = yx - y * a.wout;
    float v[9];
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int yy = net_src(y, t / 3, a.stride, a.up, a.hin), xx = net_src(x, t % 3, a.stride, a.up, a.win);
      v[t] = (yy >= 0 && xx >= 0) ? __bfloat162float(in[((size_t)n * a.hin + yy) * a.win + xx]) : 0.f;
    }
    uint32_t pk[8];
#pragma unroll
    for (int c = 0; c < 16; c += 2) {
      float r0 = 0.f, r1 = 0.f;
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        r0 = fmaf(ws[c][t], v[t], r0);
        r1 = fmaf(ws[c + 1][t], v[t], r1);
      }
      r0 = fmaxf(r0 + bs[c], 0.f);
      r1 = fmaxf(r1 + bs[c + 1], 0.f);
      const __nv_bfloat162 h2 = __floats2bfloat162_rn(r0, r1);
      pk[c / 2] = *reinterpret_cast<const uint32_t*>(&h2);
    }
    uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(a.out) + (size_t)p * 16);
    dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
  }
}

// Last layer of the inference forward (16 -> 2 channels, 3 x 3, no ReLU) on
// the CUDA cores, from channel-last BF16 input (tap-major weights) to the
// FP32 [B][2][h][w] output.  Thread = one output pixel.
__global__ void __launch_bounds__(256) k_conv_last_nhwc(ConvArgs a) {
  __shared__ float ws[2][9][16];
  for (int i = threadIdx.x; i < 2 * 9 * 16; i += blockDim.x) ws[i / 144][(i / 16) % 9][i % 16] = __bfloat162float(a.w[i]);
  __syncthreads();
  const __nv_bfloat16* in = reinterpret_cast<const __nv_bfloat16*>(a.in);
  const int hw = a.hout * a.wout, npix = a.B * hw;
  float* out = reinterpret_cast<float*>(a.out);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += gridDim.x * blockDim.x) {
    const int n = p / hw, yx = p - n * hw, y = yx / a.wout, x = yx - y * a.wout;
    float r0 = 0.f, r1 = 0.f;
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      const int yy = net_src(y, t / 3, a.stride, a.up, a.hin), xx = net_src(x, t % 3, a.stride, a.up, a.win);
      if (yy < 0 || xx < 0) continue;
      const uint4* src = reinterpret_cast<const uint4*>(in + (((size_t)n * a.hin + yy) * a.win + xx) * 16);
      const uint4 q[2] = {__ldg(src), __ldg(src + 1)};
      const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(q);
#pragma unroll
      for (int c = 0; c < 16; c += 2) {
        const float2 f = __bfloat1622float2(h[c / 2]);
        r0 = fmaf(ws[0][t][c], f.x, r0);
        r0 = fmaf(ws[0][t][c + 1], f.y, r0);
        r1 = fmaf(ws[1][t][c], f.x, r1);
        r1 = fmaf(ws[1][t][c + 1], f.y, r1);
      }
    }
    out[(size_t)(n * 2) * hw + yx] = r0 + a.b[0];
    out[(size_t)(n * 2 + 1) * hw + yx] = r1 + a.b[1];
  }
}

// Tap-major copy of one layer's BF16 weights: wt[co][tap][ci] = w[co][ci][tap].
__global__ void k_perm_weights(const __nv_bfloat16* __restrict__ w, __nv_bfloat16* __restrict__ wt, int co, int ci) {
  const int n = co * ci * 9;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int o = i / (9 * ci), r = i - o * 9 * ci, t = r / ci, c = r - t * ci;
    wt[i] = w[((size_t)o * ci + c) * 9 + t];
  }
}

// Backward data: thread = one input pixel, CV_CI input channels:
//   din[n][ci][iy][ix] = sum_co sum_taps w[co][ci][t] dout[n][co][y][x]
// over the output pixels (y, x) whose tap t reads (iy, ix); multiplied by the
// previous layer's relu derivative (mask > 0) when a mask is given.
template <typename TA>
__global__ void __launch_bounds__(CV_NT) k_conv_bwd_data(ConvArgs a) {
  __shared__ __align__(16) float ws[CV_CO][9][CV_CI];
  const int tid = threadIdx.x;
  const long long npix = (long long)a.B * a.hin * a.win;
  const long long p = (long long)blockIdx.x * CV_NT + tid;
  const bool valid = p < npix;
  const int n = valid ? (int)(p / (a.hin * a.win)) : 0;
  const int iy = valid ? (int)((p / a.win) % a.hin) : 0;
  const int ix = valid ? (int)(p % a.win) : 0;
  const int ci0 = blockIdx.y * CV_CI;
  float acc[CV_CI];
#pragma unroll
  for (int c = 0; c < CV_CI; ++c) acc[c] = 0.f;
  // output rows / columns reading this input row / column, per tap (<= 2 each
  // with upsampling: the two virtual rows 2 iy and 2 iy + 1)
  int oy[3][2], ox[3][2];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      oy[d][h] = -1;
      ox[d][h] = -1;
      if (h == 1 && !a.up) continue;
      const int vy = a.up ? 2 * iy + h : iy, vx = a.up ? 2 * ix + h : ix;
      const int ty = vy + 1 - d, tx = vx + 1 - d;
      if (ty >= 0 && ty % a.stride == 0 && ty / a.stride < a.hout) oy[d][h] = ty / a.stride;
      if (tx >= 0 && tx % a.stride == 0 && tx / a.stride < a.wout) ox[d][h] = tx / a.stride;
    }
  }
  for (int co0 = 0; co0 < a.co; co0 += CV_CO) {
    __syncthreads();
    for (int i = tid; i < CV_CO * 9 * CV_CI; i += CV_NT) {
      const int c = i / (9 * CV_CI), t = (i / CV_CI) % 9, ci = i % CV_CI;
      ws[c][t][ci] = (co0 + c < a.co && ci0 + ci < a.ci)
                         ? __bfloat162float(a.w[((size_t)(co0 + c) * a.ci + ci0 + ci) * 9 + t])
                         : 0.f;
    }
    __syncthreads();
    if (valid) {
      const int nco = min(CV_CO, a.co - co0);
      for (int c = 0; c < nco; ++c) {
        const float* g = a.dout + ((size_t)n * a.co + co0 + c) * a.hout * a.wout;
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
          for (int hy = 0; hy < 2; ++hy) {
            if (oy[dy][hy] < 0) continue;
#pragma unroll
            for (int dx = 0; dx < 3; ++dx)
#pragma unroll
              for (int hx = 0; hx < 2; ++hx) {
                if (ox[dx][hx] < 0) continue;
                const float gv = g[oy[dy][hy] * a.wout + ox[dx][hx]];
                const float4* wv = reinterpret_cast<const float4*>(&ws[c][dy * 3 + dx][0]);
#pragma unroll
                for (int q = 0; q < CV_CI / 4; ++q) {
                  const float4 w4 = wv[q];
                  acc[4 * q + 0] = fmaf(w4.x, gv, acc[4 * q + 0]);
                  acc[4 * q + 1] = fmaf(w4.y, gv, acc[4 * q + 1]);
                  acc[4 * q + 2] = fmaf(w4.z, gv, acc[4 * q + 2]);
                  acc[4 * q + 3] = fmaf(w4.w, gv, acc[4 * q + 3]);
                }
              }
          }
      }
    }
  }
  if (!valid) return;
#pragma unroll
  for (int c = 0; c < CV_CI; ++c) {
    if (ci0 + c >= a.ci) continue;
    const size_t o = (((size_t)n * a.ci + ci0 + c) * a.hin + iy) * a.win + ix;
    float r = acc[c];
    if (a.mask && !(ldact(reinterpret_cast<const TA*>(a.mask), o) > 0.f)) r = 0.f;
    a.din[o] = r;
  }
}

// Backward weights, stage 1: CTA = (co, 4 input channels, chunk of output
// pixels); per-thread FP32 sums, fixed-order block reduction, one partial per
// chunk.
constexpr int BW_CI = 4, BW_CHUNK = 4096;
template <typename TA>
__global__ void __launch_bounds__(CV_NT) k_conv_bwd_w(ConvArgs a) {
  const TA* in = reinterpret_cast<const TA*>(a.in);
  __shared__ float red[CV_NT / 32][BW_CI * 9];
  const int tid = threadIdx.x;
  const int nciq = (a.ci + BW_CI - 1) / BW_CI;
  const int co = blockIdx.x / nciq, ci0 = (blockIdx.x % nciq) * BW_CI;
  const long long npix = (long long)a.B * a.hout * a.wout;
  const long long p0 = (long long)blockIdx.y * BW_CHUNK;
  const long long p1 = min(npix, p0 + BW_CHUNK);
  float acc[BW_CI][9];
#pragma unroll
  for (int c = 0; c < BW_CI; ++c)
#pragma unroll
    for (int t = 0; t < 9; ++t) acc[c][t] = 0.f;
  for (long long p = p0 + tid; p < p1; p += CV_NT) {
    const int n = (int)(p / (a.hout * a.wout));
    const int y = (int)((p / a.wout) % a.hout), x = (int)(p % a.wout);
    const float g = a.dout[(((size_t)n * a.co + co) * a.hout + y) * a.wout + x];
    int sy[3], sx[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      sy[d] = net_src(y, d, a.stride, a.up, a.hin);
      sx[d] = net_src(x, d, a.stride, a.up, a.win);
    }
#pragma unroll
    for (int c = 0; c < BW_CI; ++c) {
      if (ci0 + c >= a.ci) continue;
      const TA* src = in + ((size_t)n * a.ci + ci0 + c) * a.hin * a.win;
#pragma unroll
      for (int dy = 0; dy < 3; ++dy)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          if (sy[dy] < 0 || sx[dx] < 0) continue;
          acc[c][dy * 3 + dx] = fmaf(g, ldact(src, (size_t)sy[dy] * a.win + sx[dx]), acc[c][dy * 3 + dx]);
        }
    }
  }
  // warp tree, then warps in order
  const int lane = tid & 31, wp = tid >> 5;
#pragma unroll
  for (int c = 0; c < BW_CI; ++c)
#pragma unroll
    for (int t = 0; t < 9; ++t) {
      float v = acc[c][t];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) red[wp][c * 9 + t] = v;
    }
  __syncthreads();
  if (tid < BW_CI * 9) {
    float s = 0.f;
    for (int w = 0; w < CV_NT / 32; ++w) s += red[w][tid];
    const int c = tid / 9, t = tid % 9;
    if (ci0 + c < a.ci) a.wpart[(((size_t)blockIdx.y * a.co + co) * a.ci + ci0 + c) * 9 + t] = s;
  }
}

// Backward weights, stage 2: sum the chunk partials in order.
__global__ void k_sum_chunks(const float* __restrict__ part, int nchunk, size_t n, float* __restrict__ out) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int c = 0; c < nchunk; ++c) s += part[(size_t)c * n + i];
    out[i] = s;
  }
}

// The same sums for few weights and many chunks: a warp per weight, lane l
// adding chunks l, l + 32, ... in order, then a fixed butterfly across the
// lanes (deterministic; the serial per-thread loop is a long latency chain
// there).
__global__ void __launch_bounds__(256) k_sum_chunks_warp(const float* __restrict__ part, int nchunk, size_t n,
                                                         float* __restrict__ out) {
  const size_t i = (size_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  float s = 0.f;
  for (int c = lane; c < nchunk; c += 32) s += part[(size_t)c * n + i];
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
  if (lane == 0) out[i] = s;
}

// Bias gradient, stage 1: CTA (channel, slice) sums its slice of the
// channel's B x hw deltas (FP32 per thread, FP64 block sum) into
// part[slice][channel]; stage 2 adds the slices in order.
__global__ void __launch_bounds__(CV_NT) k_bias_grad_part(const float* __restrict__ dout, int B, int co, int hw,
                                                           int nslice, double* __restrict__ part) {
  __shared__ double red[32];
  const int c = blockIdx.x, sl = blockIdx.y;
  const int tot = B * hw;
  const int i0 = (int)((long long)tot * sl / nslice), i1 = (int)((long long)tot * (sl + 1) / nslice);
  float s = 0.f;
  for (int i = i0 + threadIdx.x; i < i1; i += CV_NT) {
    const int n = i / hw, r = i - n * hw;
    s += dout[((size_t)n * co + c) * hw + r];
  }
  const double t = block_sum_d<CV_NT>((double)s, red);
  if (threadIdx.x == 0) part[(size_t)sl * co + c] = t;
}

__global__ void k_bias_grad_sum(const double* __restrict__ part, int nslice, int co, float* __restrict__ db) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= co) return;
  double s = 0.0;
  for (int sl = 0; sl < nslice; ++sl) s += part[(size_t)sl * co + c];
  db[c] = (float)s;
}

// Loss L = sum (out - target)^2 / (B * 2 * 64 * 64) and its gradient.
__global__ void __launch_bounds__(CV_NT) k_net_loss(const float* __restrict__ out, const float* __restrict__ tgt,
                                                     size_t n, float scale, float* __restrict__ dout,
                                                     double* __restrict__ part) {
  __shared__ double red[32];
  double s = 0.0;
  for (size_t i = blockIdx.x * (size_t)CV_NT + threadIdx.x; i < n; i += (size_t)gridDim.x * CV_NT) {
    const float d = out[i] - tgt[i];
    dout[i] = 2.f * d * scale;
    s += (double)d * d;
  }
  const double t = block_sum_d<CV_NT>(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t * scale;
}

// AdamW on the FP32 master parameters; refreshes the BF16 weight copy.
struct AdamArgs {
  float* p;
  const float* g;
  float* m;
  float* v;
  __nv_bfloat16* wb;     // BF16 copy (weights only; NULL entries skipped via is_w)
  __nv_bfloat16* wt;     // tap-major BF16 copy, or NULL
  const unsigned char* is_w;
  const int* wb_index;   // position of the parameter in the BF16 copy
  const int* wt_index;   // ... and in the tap-major copy
  size_t n;
  float lr, b1, b2, eps, wd, c1, c2;  // c1 = 1 - b1^t, c2 = 1 - b2^t
};

__global__ void k_adam(AdamArgs a) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < a.n; i += (size_t)gridDim.x * blockDim.x) {
    const float g = a.g[i];
    const float m = a.b1 * a.m[i] + (1.f - a.b1) * g;
    const float v = a.b2 * a.v[i] + (1.f - a.b2) * g * g;
    a.m[i] = m;
    a.v[i] = v;
    float p = a.p[i];
    p -= a.lr * ((m / a.c1) / (sqrtf(v / a.c2) + a.eps) + (a.is_w[i] ? a.wd * p : 0.f));
    a.p[i] = p;
    if (a.is_w[i]) {
      const __nv_bfloat16 h = __float2bfloat16_rn(p);
      a.wb[a.wb_index[i]] = h;
      if (a.wt) a.wt[a.wt_index[i]] = h;
    }
  }
}

// Network input: x = log(1 + max(I, 0)) / 10 (BF16, or FP32 in verification
// mode), from detector-centred
// FP32 intensities (src_fft == 0) or from stored FFT-order amplitudes sqrt(I)
// (src_fft == 1; masked pixels count as 0).
template <typename TA>
__global__ void k_net_input(const void* __restrict__ src, int src_fft, int istore, const float* __restrict__ scale,
                            int j0, int B, int M, TA* __restrict__ x) {
  const size_t MM = (size_t)M * M;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)B * MM;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t b = i / MM;
    const int y = (int)((i % MM) / M), xx = (int)(i % M);
    float I;
    if (!src_fft) {
      I = reinterpret_cast<const float*>(src)[i];
    } else {
      const size_t k = (j0 + b) * MM + (size_t)((y + M / 2) % M) * M + (xx + M / 2) % M;
      float a;
      if (istore == 0) a = reinterpret_cast<const float*>(src)[k];
      else if (istore == 1) a = __half2float(reinterpret_cast<const __half*>(src)[k]) * scale[j0 + b];
      else a = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(src)[k]) * scale[j0 + b];
      I = a > 0.f ? a * a : 0.f;
    }
    stact(x, i, log1pf(fmaxf(I, 0.f)) * 0.1f);
  }
}

// Training targets: amplitude and phase of the central 64 x 64 object patch
// of each position, [J][2][64][64].
__global__ void k_patch_targets(const float2* __restrict__ O, int nx, const int2* __restrict__ pos, int J, int M,
                                float* __restrict__ out) {
  const int c0 = (M - NET_OUT) / 2;
  const size_t per = (size_t)NET_OUT * NET_OUT;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (size_t)J * per;
       i += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(i / per);
    const int y = (int)((i % per) / NET_OUT), x = (int)(i % NET_OUT);
    const int2 p = pos[j];
    const float2 o = O[(size_t)(p.x + c0 + y) * nx + p.y + c0 + x];
    out[(size_t)j * 2 * per + (size_t)y * NET_OUT + x] = sqrtf(cabs2(o));
    out[(size_t)j * 2 * per + per + (size_t)y * NET_OUT + x] = atan2f(o.y, o.x);
  }
}

// Stitch predicted central patches into the object: each pixel covered by at
// least one patch becomes the mean of amp * exp(i phase) over the patches that
// cover it; other pixels keep their value.  Tile-owned over the positions'
// CSR lists (deterministic).
__global__ void __launch_bounds__(256) k_stitch(float2* __restrict__ O, int ny, int nx, int ntx,
                                                 const int* __restrict__ tile_ptr, const int* __restrict__ tile_list,
                                                 const int2* __restrict__ pos, int M, const float* __restrict__ pred,
                                                 int tile_y, int tile_x) {
  const int tile = blockIdx.x;
  const int ty0 = (tile / ntx) * tile_y, tx0 = (tile % ntx) * tile_x;
  const int c0 = (M - NET_OUT) / 2;
  const size_t per = (size_t)NET_OUT * NET_OUT;
  for (int e = threadIdx.x; e < tile_y * tile_x; e += 256) {
    const int y = ty0 + e / tile_x, x = tx0 + e % tile_x;
    if (y >= ny || x >= nx) continue;
    float2 s = make_float2(0.f, 0.f);
    int cnt = 0;
    for (int q = tile_ptr[tile]; q < tile_ptr[tile + 1]; ++q) {
      const int j = tile_list[q];
      const int2 p = pos[j];
      const int uy = y - p.x - c0, ux = x - p.y - c0;
      if (uy < 0 || uy >= NET_OUT || ux < 0 || ux >= NET_OUT) continue;
      const float amp = pred[(size_t)j * 2 * per + (size_t)uy * NET_OUT + ux];
      const float ph = pred[(size_t)j * 2 * per + per + (size_t)uy * NET_OUT + ux];
      float sn, cs;
      sincosf(ph, &sn, &cs);
      s.x += amp * cs;
      s.y += amp * sn;
      ++cnt;
    }
    if (cnt) O[(size_t)y * nx + x] = cscale(s, 1.f / cnt);
  }
}

}  // namespace ptycho

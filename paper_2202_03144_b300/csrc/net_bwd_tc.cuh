// Backward passes of the warm-start network on the tensor cores (BF16
// operands, FP32 accumulation in tensor memory), the transposes of the
// forward implicit GEMM (k_conv_fwd_tc):
//
//   weight gradient  dW[co][ci, tap] = sum_p dY[p][co] X[p][ci, tap],
//                    p over the output pixels of the batch: M = output
//                    channels, N = a tile of 144 = 9 taps x 16 input channels
//                    (column n = tap * 16 + channel), K = pixels in chunks of
//                    64; the pixel range is split over CTAs and the FP32
//                    partial tiles are summed in order afterwards
//                    (k_sum_chunks: deterministic);
//   data gradient    dX[q][ci] = sum_k G[q][k] Wt[ci][k],  k = tap * co + c,
//                    q over the input pixels: G gathers the output deltas
//                    that read pixel q through tap (zero-dilated for stride
//                    2; the two virtual rows / columns of the nearest x2
//                    upsampling summed), Wt[ci][k] = W[c][ci][tap]; the
//                    previous layer's ReLU derivative is applied in the
//                    epilogue (or in the in-order split-K reduction).
//
// Tap-major order (the tap outside the channel) lets a thread stage eight
// operand values of one tap and eight channels with one set of pixel
// offsets, held in registers (weight gradient) or loaded once per group of
// eight (data gradient), instead of recomputing the source coordinates for
// every value.
//
// Both stage their operands through two shared-memory stages in the K-major
// no-swizzle layout of tc.cuh (core matrices of 8 rows x 16 bytes), with the
// tensor cores working on one stage while the 128 threads fill the other.
// The deltas are FP32 in memory and rounded to BF16 as operands.
#pragma once
#include <cuda_bf16.h>

#include "net.cuh"
#include "tc.cuh"

namespace ptycho {

constexpr int BW_NT = 144;   // weight-gradient N tile: 16 input channels x 9 taps
constexpr int BW_NT1 = 16;   // ... for a one-channel input: the 9 taps, padded
constexpr int BW_KC = 64;    // pixels per K chunk
template <int NT>
constexpr size_t bw_tc_smem() {
  // two (A: 128 x 64, B: NT x 64) BF16 stages, mbarriers, tensor-memory slot
  return 2 * ((size_t)128 * BW_KC * 2 + (size_t)NT * BW_KC * 2) + 64;
}
// The launch asks for more at N = 144: a CTA holds 256 tensor-memory
// columns, so at most two may share an SM's 512 (a third would wait in its
// allocation).  The one-channel tile holds 32 columns: six CTAs per SM, by
// shared memory.
template <int NT>
constexpr size_t bw_tc_smem_launch() { return NT == BW_NT ? 80 * 1024 : bw_tc_smem<NT>(); }
static_assert(bw_tc_smem<BW_NT>() <= bw_tc_smem_launch<BW_NT>() && 3 * bw_tc_smem_launch<BW_NT>() > 228 * 1024,
              "two CTAs per SM");

// 8 floats -> 8 BF16 in one 16-byte word
__device__ __forceinline__ uint4 pack8_bf16(const float* v) {
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    w[i] = *reinterpret_cast<const uint32_t*>(&h);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// The BF16 im2col values of 8 output pixels (x0 .. x0 + 7 of output row y,
// x0 a multiple of 8) for vertical tap ty and the three horizontal taps, as
// w[tx][4] (value e in half e % 2 of word e / 2, as pack8_bf16 lays them
// out), read from one source plane with the coordinates of net_src:
//   stride 1:   source columns x0 - 1 .. x0 + 8: the 8 aligned values and the
//               two neighbours, each tap a shift by one value;
//   stride 2:   source columns 2 x0 - 1 .. 2 x0 + 15: 16 aligned values and
//               the left neighbour, taps 0 / 2 the odd values, tap 1 the even;
//   upsampling: source columns x0 / 2 - 1 .. x0 / 2 + 4: 4 aligned values and
//               the two neighbours, each repeated twice.
// Values outside the source are zero, as is everything when !pin.
__device__ __forceinline__ void bw_row_taps(const ConvArgs& a, const unsigned short* plane, bool pin, int y, int x0,
                                            int ty, uint32_t (&w)[3][4]) {
  int sy;
  bool ok;
  if (a.up) {
    const int vy = y + ty - 1;
    ok = pin && vy >= 0 && vy < 2 * a.hin;
    sy = vy >> 1;
  } else {
    sy = a.stride * y + ty - 1;
    ok = pin && sy >= 0 && sy < a.hin;
  }
  const unsigned short* row = plane + (size_t)(ok ? sy : 0) * a.win;
  if (a.up) {
    const int c = x0 >> 1;
    const uint2 q = ok ? __ldg(reinterpret_cast<const uint2*>(row + c)) : make_uint2(0u, 0u);
    const uint32_t L = (ok && x0 > 0) ? (uint32_t)__ldg(row + c - 1) : 0u;
    const uint32_t R = (ok && x0 + 8 < a.wout) ? (uint32_t)__ldg(row + c + 4) : 0u;
    w[1][0] = __byte_perm(q.x, q.x, 0x1010);
    w[1][1] = __byte_perm(q.x, q.x, 0x3232);
    w[1][2] = __byte_perm(q.y, q.y, 0x1010);
    w[1][3] = __byte_perm(q.y, q.y, 0x3232);
    w[0][0] = __byte_perm(L, q.x, 0x5410);
    w[0][1] = q.x;
    w[0][2] = __byte_perm(q.x, q.y, 0x5432);
    w[0][3] = q.y;
    w[2][0] = q.x;
    w[2][1] = __byte_perm(q.x, q.y, 0x5432);
    w[2][2] = q.y;
    w[2][3] = __byte_perm(q.y, R, 0x5432);
  } else if (a.stride == 1) {
    const uint4 b = ok ? __ldg(reinterpret_cast<const uint4*>(row + x0)) : make_uint4(0u, 0u, 0u, 0u);
    const uint32_t L = (ok && x0 > 0) ? (uint32_t)__ldg(row + x0 - 1) << 16 : 0u;
    const uint32_t R = (ok && x0 + 8 < a.win) ? (uint32_t)__ldg(row + x0 + 8) : 0u;
    w[1][0] = b.x;
    w[1][1] = b.y;
    w[1][2] = b.z;
    w[1][3] = b.w;
    w[0][0] = __byte_perm(L, b.x, 0x5432);
    w[0][1] = __byte_perm(b.x, b.y, 0x5432);
    w[0][2] = __byte_perm(b.y, b.z, 0x5432);
    w[0][3] = __byte_perm(b.z, b.w, 0x5432);
    w[2][0] = w[0][1];
    w[2][1] = w[0][2];
    w[2][2] = w[0][3];
    w[2][3] = __byte_perm(b.w, R, 0x5432);
  } else {
    const uint4 b0 = ok ? __ldg(reinterpret_cast<const uint4*>(row + 2 * x0)) : make_uint4(0u, 0u, 0u, 0u);
    const uint4 b1 = ok ? __ldg(reinterpret_cast<const uint4*>(row + 2 * x0 + 8)) : make_uint4(0u, 0u, 0u, 0u);
    const uint32_t L = (ok && x0 > 0) ? (uint32_t)__ldg(row + 2 * x0 - 1) << 16 : 0u;
    const uint32_t W[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      w[1][i] = __byte_perm(W[2 * i], W[2 * i + 1], 0x5410);
      w[2][i] = __byte_perm(W[2 * i], W[2 * i + 1], 0x7632);
      w[0][i] = __byte_perm(i ? W[2 * i - 1] : L, W[2 * i], 0x7632);
    }
  }
}

// Weight gradient.  grid = (co tiles of 128 x k tiles of NT, pixel splits).
// Writes the FP32 partial dW of its pixel range: part[split][co][ci * 9].
// NT = BW_NT: tap-major tiles of 16 input channels; NT = BW_NT1: the
// one-channel first layer, column = tap.
template <typename TA, int NT>
__global__ void __launch_bounds__(128) k_conv_bwd_w_tc(ConvArgs a, int nsplit, int* err_flag) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr size_t ABYTES = (size_t)128 * BW_KC * 2, BBYTES = (size_t)NT * BW_KC * 2;
  unsigned char* stage[2] = {smem_raw, smem_raw + ABYTES + BBYTES};
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + 2 * (ABYTES + BBYTES));
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  constexpr uint32_t LBO = 128, SBO = (BW_KC / 8) * 128;
  constexpr uint32_t NCOLS = NT <= 32 ? 32 : 256;
  const TA* in = reinterpret_cast<const TA*>(a.in);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int KW = a.ci * 9;
  const int nkt = (KW + NT - 1) / NT;
  const int co0 = (blockIdx.x / nkt) * 128, k0 = (blockIdx.x % nkt) * NT;
  const int hw = a.hout * a.wout;
  const long long npix = (long long)a.B * hw;
  const long long nchunk = (npix + BW_KC - 1) / BW_KC;
  const long long c_begin = nchunk * blockIdx.y / nsplit, c_end = nchunk * (blockIdx.y + 1) / nsplit;
  // rows past the output channels / past the input channels stay zero:
  // written once
  const int rows_a = min(128, a.co - co0);
  // B rows n = tap * 16 + cl: this thread stages channel ci0 + cl (the same
  // for every chunk) for all nine taps, pixel group tid % 8
  const int ci0 = k0 / 9, cl = tid >> 3;
  const int ncl = min(16, a.ci - ci0);  // input channels of this tile
  for (int i = tid; i < (int)(2 * (ABYTES + BBYTES) / 16); i += 128)
    reinterpret_cast<uint4*>(smem_raw)[i] = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    tc::mbar_init1(&bar[0]);
    tc::mbar_init1(&bar[1]);
  }
  if (warp == 0) tc::tmem_alloc(tslot, NCOLS);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = *tslot;
  constexpr uint32_t idesc = tc::idesc_bf16_f32(128, NT);
  uint32_t ph[2] = {0u, 0u};
  bool pending[2] = {false, false};
  bool ok = true;
  for (long long c = c_begin; c < c_end; ++c) {
    const int s = (int)((c - c_begin) & 1);
    if (pending[s]) {
      if (!tc::mbar_wait(&bar[s], ph[s])) ok = false;
      ph[s] ^= 1u;
      pending[s] = false;
      tc::fence_after();
    }
    unsigned char* As = stage[s];
    unsigned char* Bs = stage[s] + ABYTES;
    const long long p0 = c * BW_KC;
    // this thread's 8 pixels of the chunk: p0 + 8 g .. + 7 (g = tid % 8, the
    // same for every unit the thread stages; hw is a multiple of 8, so the
    // group lies in one image)
    const long long pg = p0 + 8 * (tid & 7);
    const bool pin = pg < npix;
    const int n = pin ? (int)(pg / hw) : 0;
    const int yx0 = pin ? (int)(pg - (long long)n * hw) : 0;
    // A: dY rows (output channels) x 64 pixels: two 16-byte loads per unit
    for (int u = tid; u < rows_a * (BW_KC / 8); u += 128) {
      const int r = u >> 3, g = u & 7;
      const int co = co0 + r;
      float v[8];
      if (pin) {
        const float4* src = reinterpret_cast<const float4*>(a.dout + ((size_t)n * a.co + co) * hw + yx0);
        const float4 q0 = __ldg(src), q1 = __ldg(src + 1);
        v[0] = q0.x, v[1] = q0.y, v[2] = q0.z, v[3] = q0.w, v[4] = q1.x, v[5] = q1.y, v[6] = q1.z, v[7] = q1.w;
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = 0.f;
      }
      *reinterpret_cast<uint4*>(As + (r >> 3) * SBO + g * LBO + (r & 7) * 16) = pack8_bf16(v);
    }
    // B: im2col rows (tap, channel) x 64 pixels, the forward's gather.  This
    // thread's 8 pixels' source rows (as plane offsets) and columns for the
    // three vertical and three horizontal taps, once per chunk (wout >= 4:
    // at most one row change inside the group); -1 outside the input.
    if (NT == BW_NT && ncl == 16 && a.wout % 8 == 0 && sizeof(TA) == 2) {
      // output rows of at least 8 pixels: the 8 pixels of a group share one
      // output row, and for each vertical tap one aligned load of the source
      // row segment (16 bytes, stride 2: 32, upsampling: 8) plus the edge
      // values yields all three horizontal taps by byte permutes
      // (bw_row_taps); the source coordinates are those of net_src
      const unsigned short* plane16 =
          reinterpret_cast<const unsigned short*>(in) + ((size_t)n * a.ci + ci0 + cl) * a.hin * a.win;
      const int y = yx0 / a.wout, x0 = yx0 - y * a.wout;
      const int g = tid & 7;
#pragma unroll
      for (int ty = 0; ty < 3; ++ty) {
        uint32_t w[3][4];
        bw_row_taps(a, plane16, pin, y, x0, ty, w);
#pragma unroll
        for (int tx = 0; tx < 3; ++tx) {
          const int r = (ty * 3 + tx) * 16 + cl;
          *reinterpret_cast<uint4*>(Bs + (r >> 3) * SBO + g * LBO + (r & 7) * 16) =
              make_uint4(w[tx][0], w[tx][1], w[tx][2], w[tx][3]);
        }
      }
    } else if (NT == BW_NT && ncl == 16) {
      const TA* plane = in + ((size_t)n * a.ci + ci0 + cl) * a.hin * a.win;
      int roff[3][8], sx[3][8];
      {
        int y = yx0 / a.wout, x = yx0 - y * a.wout;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const int sy = pin ? net_src(y, d, a.stride, a.up, a.hin) : -1;
            roff[d][e] = sy >= 0 ? sy * a.win : -1;
            sx[d][e] = pin ? net_src(x, d, a.stride, a.up, a.win) : -1;
          }
          if (++x == a.wout) {
            x = 0;
            ++y;
          }
        }
      }
      const int g = tid & 7;
#pragma unroll
      for (int t = 0; t < 9; ++t) {
        const int r = t * 16 + cl;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int ro = roff[t / 3][e], cx = sx[t % 3][e];
          v[e] = (ro >= 0 && cx >= 0) ? ldact(plane, (size_t)(ro + cx)) : 0.f;
        }
        *reinterpret_cast<uint4*>(Bs + (r >> 3) * SBO + g * LBO + (r & 7) * 16) = pack8_bf16(v);
      }
    } else {
      // fewer channels (the one-channel first layer): the (tap, channel,
      // pixel group) units spread over all threads, source coordinates per
      // value; the pixel group is tid % 8 for every unit of the thread
      int py[8], px[8];
      {
        int y = yx0 / a.wout, x = yx0 - y * a.wout;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          py[e] = y;
          px[e] = x;
          if (++x == a.wout) {
            x = 0;
            ++y;
          }
        }
      }
      for (int u = tid; u < 9 * ncl * 8; u += 128) {
        const int g = u & 7, c2 = (u >> 3) % ncl, t = (u >> 3) / ncl, ty = t / 3, tx = t - 3 * ty;
        const TA* plane = in + ((size_t)n * a.ci + ci0 + c2) * a.hin * a.win;
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          float x = 0.f;
          if (pin) {
            const int sy = net_src(py[e], ty, a.stride, a.up, a.hin), sx = net_src(px[e], tx, a.stride, a.up, a.win);
            if (sy >= 0 && sx >= 0) x = ldact(plane, (size_t)sy * a.win + sx);
          }
          v[e] = x;
        }
        const int r = t * (NT == BW_NT ? 16 : 1) + c2;  // one-channel tile: column = tap
        *reinterpret_cast<uint4*>(Bs + (r >> 3) * SBO + g * LBO + (r & 7) * 16) = pack8_bf16(v);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc::fence_before();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
#pragma unroll
      for (int kk = 0; kk < BW_KC / 16; ++kk) {
        const uint64_t ad = tc::smem_desc(As + kk * 2 * LBO, LBO, SBO);
        const uint64_t bd = tc::smem_desc(Bs + kk * 2 * LBO, LBO, SBO);
        tc::mma_bf16(tbase, ad, bd, idesc, (c > c_begin || kk > 0) ? 1u : 0u);
      }
      tc::commit(&bar[s]);
    }
    pending[s] = true;
  }
#pragma unroll
  for (int s = 0; s < 2; ++s)
    if (pending[s] && !tc::mbar_wait(&bar[s], ph[s])) ok = false;
  tc::fence_after();
  if (!ok && tid == 0) atomicExch(err_flag, 1);
  // epilogue: lane = output channel co0 + 32 warp + lane, columns = k tile
  const int co = co0 + warp * 32 + (tid & 31);
  const bool any = c_end > c_begin;
#pragma unroll 1
  for (int c0 = 0; c0 < NT; c0 += 16) {
    float v[16];
    tc::tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
    if (co < a.co) {
      if constexpr (NT == BW_NT) {
        // column c0 + j = tap * 16 + channel: a 16-column slice is one tap
        const int t = c0 >> 4;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int ci = ci0 + j;
          if (ci < a.ci) a.wpart[((size_t)blockIdx.y * a.co + co) * KW + ci * 9 + t] = any ? v[j] : 0.f;
        }
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j)  // column = tap of the one channel
          if (j < KW) a.wpart[((size_t)blockIdx.y * a.co + co) * KW + j] = any ? v[j] : 0.f;
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tbase, NCOLS);
}

// Data gradient.  grid = (input-pixel tiles of 128, K splits).  NP = input
// channels rounded up to 16.  ksplit == 1: dX (masked) straight to a.din;
// else FP32 partials part[split][ci][pixel], reduced by k_bwd_data_reduce.
constexpr int BD_KC = 64;
template <int NP>
__host__ __device__ constexpr size_t bd_tc_smem() {
  // two (A, B) stages, mbarriers and slot, the per-thread delta offsets
  // [9 taps][4 (row, column) choices][128]
  return 2 * ((size_t)128 * BD_KC * 2 + (size_t)NP * BD_KC * 2) + 64 + 36 * 128 * 4;
}

template <typename TA, int NP>
__global__ void __launch_bounds__(128) k_conv_bwd_data_tc(ConvArgs a, int ksplit, float* part, int* err_flag) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr size_t ABYTES = (size_t)128 * BD_KC * 2, BBYTES = (size_t)NP * BD_KC * 2;
  unsigned char* stage[2] = {smem_raw, smem_raw + ABYTES + BBYTES};
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + 2 * (ABYTES + BBYTES));
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  int* offs = reinterpret_cast<int*>(smem_raw + 2 * (ABYTES + BBYTES) + 64);  // [36][128]
  constexpr uint32_t LBO = 128, SBO = (BD_KC / 8) * 128;
  constexpr uint32_t NCOLS = NP < 32 ? 32 : NP;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int hwi = a.hin * a.win, hwo = a.hout * a.wout;
  const long long npix = (long long)a.B * hwi;
  const long long q = (long long)blockIdx.x * 128 + tid;  // this thread's input pixel
  const bool valid = q < npix;
  const int n = valid ? (int)(q / hwi) : 0;
  const int iyx = valid ? (int)(q - (long long)n * hwi) : 0;
  const int iy = iyx / a.win, ix = iyx - iy * a.win;
  // output rows / columns that read this input row / column through tap d
  // (two each with upsampling: the virtual rows 2 iy and 2 iy + 1)
  {
    int oy[3][2], ox[3][2];
#pragma unroll
    for (int d = 0; d < 3; ++d)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        oy[d][h] = -1;
        ox[d][h] = -1;
        if (h == 1 && !a.up) continue;
        const int vy = a.up ? 2 * iy + h : iy, vx = a.up ? 2 * ix + h : ix;
        const int ty = vy + 1 - d, tx = vx + 1 - d;
        if (valid && ty >= 0 && ty % a.stride == 0 && ty / a.stride < a.hout) oy[d][h] = ty / a.stride;
        if (valid && tx >= 0 && tx % a.stride == 0 && tx / a.stride < a.wout) ox[d][h] = tx / a.stride;
      }
    // offset of each (tap, row choice, column choice) delta in its plane, -1: none
#pragma unroll
    for (int t = 0; t < 9; ++t)
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const int yy = oy[t / 3][h >> 1], xx = ox[t % 3][h & 1];
        offs[(t * 4 + h) * 128 + tid] = (yy >= 0 && xx >= 0) ? yy * a.wout + xx : -1;
      }
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
  const int K = a.co * 9;
  const bool co8 = (a.co & 7) == 0;
  const int nchunk = (K + BD_KC - 1) / BD_KC;
  const int c_begin = (int)(((long long)nchunk * blockIdx.y) / ksplit);
  const int c_end = (int)(((long long)nchunk * (blockIdx.y + 1)) / ksplit);
  const float* dy = a.dout + (size_t)n * a.co * hwo;
  constexpr uint32_t idesc = tc::idesc_bf16_f32(128, NP);
  uint32_t ph[2] = {0u, 0u};
  bool pending[2] = {false, false};
  bool ok = true;
  for (int c = c_begin; c < c_end; ++c) {
    const int s = (c - c_begin) & 1;
    if (pending[s]) {
      if (!tc::mbar_wait(&bar[s], ph[s])) ok = false;
      ph[s] ^= 1u;
      pending[s] = false;
      tc::fence_after();
    }
    unsigned char* As = stage[s];
    unsigned char* Bs = stage[s] + ABYTES;
    const int kb = c * BD_KC;
    // A: this thread's pixel (row tid), 64 values of k = tap * co + c.
    // With co a multiple of 8 a group of eight k is one tap and eight
    // channels: its delta offsets are read once and the eight loads differ
    // by whole planes.
#pragma unroll 1
    for (int g = 0; g < BD_KC / 8; ++g) {
      float v[8];
      const int kg = kb + 8 * g;
      if (co8) {
        const int t = kg / a.co, c = kg - t * a.co;
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = 0.f;
        if (kg < K) {
          const float* pl = dy + (size_t)c * hwo;
          const int o0 = offs[(t * 4) * 128 + tid];
          if (o0 >= 0)
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = pl[(size_t)e * hwo + o0];
          if (a.up) {  // the other virtual rows / columns of the upsampling
#pragma unroll
            for (int h = 1; h < 4; ++h) {
              const int o = offs[(t * 4 + h) * 128 + tid];
              if (o >= 0)
#pragma unroll
                for (int e = 0; e < 8; ++e) v[e] += pl[(size_t)e * hwo + o];
            }
          }
        }
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int k = kg + e;
          float x = 0.f;
          if (k < K) {
            const int t = k / a.co, c = k - t * a.co;
            const float* pl = dy + (size_t)c * hwo;
            const int o0 = offs[(t * 4) * 128 + tid];
            if (o0 >= 0) x = pl[o0];
            if (a.up) {
#pragma unroll
              for (int h = 1; h < 4; ++h) {
                const int o = offs[(t * 4 + h) * 128 + tid];
                if (o >= 0) x += pl[o];
              }
            }
          }
          v[e] = x;
        }
      }
      *reinterpret_cast<uint4*>(As + (tid >> 3) * SBO + g * LBO + (tid & 7) * 16) = pack8_bf16(v);
    }
    // B: Wt rows (input channels) x 64 values of k: W[c][ci][tap]
    for (int u = tid; u < NP * (BD_KC / 8); u += 128) {
      const int r = u / (BD_KC / 8), g = u % (BD_KC / 8);
      __align__(16) __nv_bfloat16 w8[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = kb + 8 * g + e;
        const int t = k / a.co, c = k - t * a.co;
        w8[e] = (r < a.ci && k < K) ? a.w[((size_t)c * a.ci + r) * 9 + t] : __float2bfloat16_rn(0.f);
      }
      *reinterpret_cast<uint4*>(Bs + (r >> 3) * SBO + g * LBO + (r & 7) * 16) = *reinterpret_cast<const uint4*>(w8);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc::fence_before();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
#pragma unroll
      for (int kk = 0; kk < BD_KC / 16; ++kk) {
        const uint64_t ad = tc::smem_desc(As + kk * 2 * LBO, LBO, SBO);
        const uint64_t bd = tc::smem_desc(Bs + kk * 2 * LBO, LBO, SBO);
        tc::mma_bf16(tbase, ad, bd, idesc, (c > c_begin || kk > 0) ? 1u : 0u);
      }
      tc::commit(&bar[s]);
    }
    pending[s] = true;
  }
#pragma unroll
  for (int s = 0; s < 2; ++s)
    if (pending[s] && !tc::mbar_wait(&bar[s], ph[s])) ok = false;
  tc::fence_after();
  if (!ok && tid == 0) atomicExch(err_flag, 1);
  const bool any = c_end > c_begin;
  // epilogue: lane = input pixel blockIdx.x * 128 + tid, columns = ci
#pragma unroll 1
  for (int c0 = 0; c0 < NP; c0 += 16) {
    float v[16];
    tc::tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
    if (!valid) continue;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int ci = c0 + j;
      if (ci >= a.ci) continue;
      const float r = any ? v[j] : 0.f;
      if (ksplit > 1) {
        part[((size_t)blockIdx.y * a.ci + ci) * npix + q] = r;
        continue;
      }
      const size_t o = ((size_t)n * a.ci + ci) * hwi + iyx;
      float rr = r;
      if (a.mask && !(ldact(reinterpret_cast<const TA*>(a.mask), o) > 0.f)) rr = 0.f;
      a.din[o] = rr;
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tbase, NCOLS);
}

// Data gradient of a stride-2 layer, by input-pixel parity class.  An input
// pixel (iy, ix) is read by tap (dy, dx) of output (oy, ox) only where
// iy + 1 - dy = 2 oy and ix + 1 - dx = 2 ox: the even rows through dy = 1,
// the odd rows through dy = 0 and 2 (likewise for columns).  So the pixels
// of one parity class (iy % 2, ix % 2) take 1, 2, 2 or 4 taps, and a tile of
// 128 pixels of one class runs a GEMM over K = co x its taps with no zero
// rows: k = t * co + c, t the index of the tap in the class's list.
// grid = (4 classes x tiles of 128 class pixels, K splits).  The class's
// pixels are (iy, ix) = (2 my + py, 2 mx + px), my < hin / 2, mx < win / 2.
template <typename TA, int NP>
__host__ __device__ constexpr size_t bd_s2_tc_smem() {
  return 2 * ((size_t)128 * BD_KC * 2 + (size_t)NP * BD_KC * 2) + 64 + 4 * 128 * 4;
}

template <typename TA, int NP>
__global__ void __launch_bounds__(128) k_conv_bwd_data_s2_tc(ConvArgs a, int ksplit, float* part, int* err_flag) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr size_t ABYTES = (size_t)128 * BD_KC * 2, BBYTES = (size_t)NP * BD_KC * 2;
  unsigned char* stage[2] = {smem_raw, smem_raw + ABYTES + BBYTES};
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + 2 * (ABYTES + BBYTES));
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 2);
  int* offs = reinterpret_cast<int*>(smem_raw + 2 * (ABYTES + BBYTES) + 64);  // [4][128]
  constexpr uint32_t LBO = 128, SBO = (BD_KC / 8) * 128;
  constexpr uint32_t NCOLS = NP < 32 ? 32 : NP;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int hwi = a.hin * a.win, hwo = a.hout * a.wout;
  const int hh = a.hin >> 1, wh = a.win >> 1, pc = hh * wh;
  const long long ncls = (long long)a.B * pc;             // pixels per class
  const long long tiles = (ncls + 127) / 128;
  const int cls = (int)(blockIdx.x / tiles);
  const int py = cls >> 1, px = cls & 1;
  const long long qc = (long long)(blockIdx.x % tiles) * 128 + tid;
  const bool valid = qc < ncls;
  const int n = valid ? (int)(qc / pc) : 0;
  const int r = valid ? (int)(qc - (long long)n * pc) : 0;
  const int iy = 2 * (r / wh) + py, ix = 2 * (r % wh) + px;
  const long long q = (long long)n * hwi + (long long)iy * a.win + ix;  // pixel index in the batch
  // the class's taps: rows dy = 1 (even iy) or 0, 2 (odd); columns likewise
  const int nty = py ? 2 : 1, ntx = px ? 2 : 1, ntap = nty * ntx;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    int o = -1;
    if (t < ntap && valid) {
      const int dy = py ? 2 * (t / ntx) : 1, dx = px ? 2 * (t % ntx) : 1;
      const int oy = (iy + 1 - dy) >> 1, ox = (ix + 1 - dx) >> 1;  // exact: the parity matches
      if (iy + 1 - dy >= 0 && oy < a.hout && ix + 1 - dx >= 0 && ox < a.wout) o = oy * a.wout + ox;
    }
    offs[t * 128 + tid] = o;
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
  const int K = a.co * ntap;  // co is a multiple of 8: a group of eight k is one tap
  const int nchunk = (K + BD_KC - 1) / BD_KC;
  const int c_begin = (int)(((long long)nchunk * blockIdx.y) / ksplit);
  const int c_end = (int)(((long long)nchunk * (blockIdx.y + 1)) / ksplit);
  const float* dy_n = a.dout + (size_t)n * a.co * hwo;
  constexpr uint32_t idesc = tc::idesc_bf16_f32(128, NP);
  uint32_t ph[2] = {0u, 0u};
  bool pending[2] = {false, false};
  bool ok = true;
  for (int c = c_begin; c < c_end; ++c) {
    const int s = (c - c_begin) & 1;
    if (pending[s]) {
      if (!tc::mbar_wait(&bar[s], ph[s])) ok = false;
      ph[s] ^= 1u;
      pending[s] = false;
      tc::fence_after();
    }
    unsigned char* As = stage[s];
    unsigned char* Bs = stage[s] + ABYTES;
    const int kb = c * BD_KC;
    // A: this thread's pixel, 64 values of k: eight groups of one tap and
    // eight channels, all loads of the chunk in flight together
#pragma unroll
    for (int g = 0; g < BD_KC / 8; ++g) {
      float v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = 0.f;
      const int kg = kb + 8 * g;
      if (kg < K) {
        const int t = kg / a.co, ch = kg - t * a.co;
        const int o = offs[t * 128 + tid];
        if (o >= 0) {
          const float* pl = dy_n + (size_t)ch * hwo + o;
#pragma unroll
          for (int e = 0; e < 8; ++e) v[e] = pl[(size_t)e * hwo];
        }
      }
      *reinterpret_cast<uint4*>(As + (tid >> 3) * SBO + g * LBO + (tid & 7) * 16) = pack8_bf16(v);
    }
    // B: Wt rows (input channels) x 64 values of k: W[c][ci][tap of t]
    for (int u = tid; u < NP * (BD_KC / 8); u += 128) {
      const int rr = u / (BD_KC / 8), g = u % (BD_KC / 8);
      __align__(16) __nv_bfloat16 w8[8];
      const int kg = kb + 8 * g;
      const int t = kg / a.co, ch = kg - t * a.co;
      const int tap = (py ? 2 * (t / ntx) : 1) * 3 + (px ? 2 * (t % ntx) : 1);
#pragma unroll
      for (int e = 0; e < 8; ++e)
        w8[e] = (rr < a.ci && kg < K) ? a.w[((size_t)(ch + e) * a.ci + rr) * 9 + tap] : __float2bfloat16_rn(0.f);
      *reinterpret_cast<uint4*>(Bs + (rr >> 3) * SBO + g * LBO + (rr & 7) * 16) = *reinterpret_cast<const uint4*>(w8);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc::fence_before();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
#pragma unroll
      for (int kk = 0; kk < BD_KC / 16; ++kk) {
        const uint64_t ad = tc::smem_desc(As + kk * 2 * LBO, LBO, SBO);
        const uint64_t bd = tc::smem_desc(Bs + kk * 2 * LBO, LBO, SBO);
        tc::mma_bf16(tbase, ad, bd, idesc, (c > c_begin || kk > 0) ? 1u : 0u);
      }
      tc::commit(&bar[s]);
    }
    pending[s] = true;
  }
#pragma unroll
  for (int s = 0; s < 2; ++s)
    if (pending[s] && !tc::mbar_wait(&bar[s], ph[s])) ok = false;
  tc::fence_after();
  if (!ok && tid == 0) atomicExch(err_flag, 1);
  const bool any = c_end > c_begin;
  const long long npix = (long long)a.B * hwi;
#pragma unroll 1
  for (int c0 = 0; c0 < NP; c0 += 16) {
    float v[16];
    tc::tmem_ld16(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
    if (!valid) continue;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int ci = c0 + j;
      if (ci >= a.ci) continue;
      const float rv = any ? v[j] : 0.f;
      if (ksplit > 1) {
        part[((size_t)blockIdx.y * a.ci + ci) * npix + q] = rv;
        continue;
      }
      const size_t o = ((size_t)n * a.ci + ci) * hwi + (size_t)iy * a.win + ix;
      float rr = rv;
      if (a.mask && !(ldact(reinterpret_cast<const TA*>(a.mask), o) > 0.f)) rr = 0.f;
      a.din[o] = rr;
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tbase, NCOLS);
}

// Split-K epilogue of the data gradient: the partials summed in order, the
// previous layer's ReLU derivative applied, into a.din [B][ci][h][w].
template <typename TA>
__global__ void k_bwd_data_reduce(ConvArgs a, int ksplit, const float* __restrict__ part) {
  const long long hwi = (long long)a.hin * a.win, npix = a.B * hwi;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npix * a.ci;
       i += (long long)gridDim.x * blockDim.x) {
    const int ci = (int)(i / npix);
    const long long q = i % npix;
    float r = 0.f;
    for (int s = 0; s < ksplit; ++s) r += part[((size_t)s * a.ci + ci) * npix + q];
    const int n = (int)(q / hwi);
    const size_t o = ((size_t)n * a.ci + ci) * hwi + (q % hwi);
    if (a.mask && !(ldact(reinterpret_cast<const TA*>(a.mask), o) > 0.f)) r = 0.f;
    a.din[o] = r;
  }
}

}  // namespace ptycho

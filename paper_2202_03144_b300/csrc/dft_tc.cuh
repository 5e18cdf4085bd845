// Fused Fourier step with the 2-D DFT on the tensor cores (64 x 64 detector,
// one probe mode): every 1-D transform of a position is one matrix product
// with the 64-point DFT matrix, in BF16 with a three-term split and FP32
// accumulation in tensor memory.
//
// Real form.  A length-64 complex DFT y = W x (W_fr = exp(-2 pi i f r / 64))
// is the real 128 x 128 product
//     [y_re; y_im] = [[C, S], [-S, C]] [x_re; x_im],  C = cos, S = sin of
// 2 pi f r / 64.  This matrix is the MMA's A operand (M = 128 rows: the real
// and imaginary parts of the 64 outputs); the B operand holds the 64 input
// vectors of one stage (N = 64 rows of K = 128: real parts, then imaginary
// parts), so D = A B^T gives, in tensor-memory lane (ri, f) and column n, the
// real (ri = 0) or imaginary (ri = 1) part of output f of input vector n.
//
// Split precision.  Every value v (matrix entry and data) is v_hi + v_lo
// with v_hi = v rounded to BF16 and v_lo = (v - v_hi) rounded to BF16; each
// product takes the three terms hi*hi + lo*hi + hi*lo (the lo*lo term, about
// 2^-18 of the product, is dropped), accumulated in FP32: about 17
// significant bits per stage instead of FP32's 24.
//
// Data flow of one position (128 threads; thread t reads tensor-memory lane
// t, i.e. (ri, f) = (t / 64, t % 64)):
//   prologue      B[c][(ri, r)] = x[r][c], x = P O_j (DM: 2 P O_j - psi)
//   stage 1       D1[(ri, f)][c]  = Y[f][c]       (column transforms)
//   stage 2       B[f][(ri, c)] = Y[f][c]: thread (ri, f) holds row f's ri
//                 part; D2[(ri, g)][f] = Z[f][g]  (row transforms)
//   projection    the two parts of Z[f][g] meet through shared memory; the
//                 detector-plane factor of the mode (as in the FFT kernels)
//                 gives D = factor Z / M^2
//   stages 3, 4   the inverse transforms as forward ones on conjugated data
//                 (F^-1 z = conj(F conj z) / M^2): B = conj(D) column-wise,
//                 then the raw stage-3 output row-wise; chi = conj(D4)
//   epilogue      thread (ri, q) holds the ri part of chi[r][q] for all r:
//                 the residual (LSQML), or phi + chi (DM), to global memory.
// Error and forward-model passes stop after the projection.
//
// One CTA walks positions with a stride of the grid (persistent; the DFT
// matrix is copied into shared memory once).  Shared memory: the split
// matrix (64 KB) and one B staging tile (32 KB, also the exchange buffer of
// the projection): two CTAs per SM.  Tensor memory: 64 columns per CTA.
#pragma once
#include <cuda_bf16.h>

#include "fourier3.cuh"
#include "tc.cuh"

namespace ptycho {

constexpr int TC64_NT = 128;
constexpr uint32_t TC64_LBO = 128, TC64_SBO = 2048;          // K-major, no swizzle, K = 128
constexpr size_t TC64_AMAT = 128 * 128 * 2;                   // one term of the DFT matrix
constexpr size_t TC64_BST = 64 * 128 * 2;                     // one term of a B tile
constexpr size_t TC64_SMEM = 2 * TC64_AMAT + 2 * TC64_BST + 64;

// byte offset of element (row, k) in a K-major no-swizzle operand with K = 128
__host__ __device__ __forceinline__ uint32_t tc64_off(int row, int k) {
  return (uint32_t)((row >> 3) * TC64_SBO + (k >> 3) * TC64_LBO + (row & 7) * 16 + (k & 7) * 2);
}

// hi / lo BF16 pairs of two floats (hi rounded half away from zero in the
// 16 dropped bits, lo = the exact remainder rounded to nearest)
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const uint32_t ua = (__float_as_uint(a) + 0x8000u) & 0xFFFF0000u;
  const uint32_t ub = (__float_as_uint(b) + 0x8000u) & 0xFFFF0000u;
  hi = __byte_perm(ua, ub, 0x7632);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - __uint_as_float(ua), b - __uint_as_float(ub));
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Eight consecutive K values of B row `row` starting at k0 (a multiple of 8):
// both terms, one 16-byte store each.
__device__ __forceinline__ void put8(unsigned char* Bst, int row, int k0, const float* v) {
  uint4 h, l;
  split2(v[0], v[1], h.x, l.x);
  split2(v[2], v[3], h.y, l.y);
  split2(v[4], v[5], h.z, l.z);
  split2(v[6], v[7], h.w, l.w);
  const uint32_t o = tc64_off(row, k0);
  *reinterpret_cast<uint4*>(Bst + o) = h;
  *reinterpret_cast<uint4*>(Bst + TC64_BST + o) = l;
}

// Thread 0: D = A_hi B_hi + A_lo B_hi + A_hi B_lo (K = 128 in steps of 16),
// then the completion is signalled on bar.
__device__ __forceinline__ void tc64_mma(uint32_t tmem, const unsigned char* Am, const unsigned char* Bst,
                                         uint64_t* bar) {
  constexpr uint32_t idesc = tc::idesc_bf16_f32(128, 64);
  const unsigned char* As[3] = {Am, Am + TC64_AMAT, Am};
  const unsigned char* Bs[3] = {Bst, Bst, Bst + TC64_BST};
#pragma unroll
  for (int t = 0; t < 3; ++t)
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const uint64_t ad = tc::smem_desc(As[t] + kk * 2 * TC64_LBO, TC64_LBO, TC64_SBO);
      const uint64_t bd = tc::smem_desc(Bs[t] + kk * 2 * TC64_LBO, TC64_LBO, TC64_SBO);
      tc::mma_bf16(tmem, ad, bd, idesc, (t > 0 || kk > 0) ? 1u : 0u);
    }
  tc::commit(bar);
}

// Warp-wide load of 32 consecutive FP32 columns of this warp's lanes.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ri part of one complex value
__device__ __forceinline__ float cpart(float2 z, int ri) { return ri ? z.y : z.x; }

template <int MODE_T = -1, int IST_T = -1>
__global__ void __launch_bounds__(TC64_NT, 2) k_fourier_tc64(Fourier2Args a, const unsigned char* dftm, int err_c) {
  constexpr int M = 64;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* Am = smem_raw;                    // split DFT matrix
  unsigned char* Bst = smem_raw + 2 * TC64_AMAT;   // B tile (hi, lo) / projection exchange
  float* xch = reinterpret_cast<float*>(Bst);      // [64 values][128 threads]
  uint64_t* bar = reinterpret_cast<uint64_t*>(Bst + 2 * TC64_BST);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  double* red = reinterpret_cast<double*>(tslot + 2);  // [4 warps][2]

  const int tid = threadIdx.x, warp = tid >> 5;
  const int ri = tid >> 6, idx = tid & 63;  // tensor-memory lane (ri, idx)
  const int mode = MODE_T >= 0 ? MODE_T : a.mode;
  const bool inverse = mode != FM_ERR && mode != FM_SIM;
  constexpr float inv = 1.0f / (float)(M * M);

  // the split matrix, once per CTA
  for (int i = tid; i < (int)(2 * TC64_AMAT / 16); i += TC64_NT)
    reinterpret_cast<uint4*>(Am)[i] = __ldg(reinterpret_cast<const uint4*>(dftm) + i);
  if (tid == 0) tc::mbar_init1(bar);
  if (warp == 0) tc::tmem_alloc(tslot, 64);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t tlane = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's lanes, column 0
  uint32_t ph = 0;
  bool ok = true;
  // stage boundary: the B tile written by every thread -> tensor cores; the
  // product's completion -> this thread's 64 columns of its lane
  auto stage = [&](float* d) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc::fence_before();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      tc64_mma(tmem, Am, Bst, bar);
    }
    if (!tc::mbar_wait(bar, ph)) ok = false;
    ph ^= 1u;
    tc::fence_after();
    tmem_ld32(tlane, d);
    tmem_ld32(tlane + 32, d + 32);
  };

  float d[64];
  for (int jj = blockIdx.x; jj < a.nj; jj += gridDim.x) {
    const int j = a.j0 + jj;
    const float2* Pj = a.pbin ? a.P + (size_t)__ldg(a.pbin + j) * (M * M) : a.P;
    const int2 p = a.pos[j];
    // ---- prologue: thread (h, c) = rows r in [32 h, 32 h + 32) of column c
    {
      const int c = idx, h = ri;
      const float2* orow = a.O + (size_t)(p.x + 32 * h) * a.nx + p.y + c;
      const float2* prow = Pj + (size_t)(32 * h) * M + c;
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        float re[8], im[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int r = 8 * g + e;
          float2 x = cmul(__ldg(prow + (size_t)r * M), __ldg(orow + (size_t)r * a.nx));
          if (mode == FM_DM)
            x = csub(cscale(x, 2.f), a.X[((size_t)(j - a.xoff) * M + 32 * h + r) * M + c]);
          re[e] = x.x;
          im[e] = x.y;
        }
        put8(Bst, c, 32 * h + 8 * g, re);
        put8(Bst, c, 64 + 32 * h + 8 * g, im);
      }
    }
    stage(d);  // D1: column transforms, d[c] = ri part of Y[idx][c]
#pragma unroll
    for (int g = 0; g < 8; ++g) put8(Bst, idx, 64 * ri + 8 * g, d + 8 * g);
    stage(d);  // D2: d[f] = ri part of Z[f][idx] (FFT order: ky = f, kx = idx)
    // ---- projection: the other part of each value through shared memory
    __syncthreads();  // every thread's stage-2 B rows were read by the finished product
#pragma unroll
    for (int f = 0; f < 64; ++f) xch[f * TC64_NT + tid] = d[f];
    __syncthreads();
    float scale = 1.f;
    const int istore = IST_T >= 0 ? IST_T : a.istore;
    if (mode != FM_SIM && istore != 0) scale = __ldg(a.amp_scale + j);
    float en = 0.f, ed = 0.f;
#pragma unroll
    for (int f = 0; f < 64; ++f) {
      const float other = xch[f * TC64_NT + (tid ^ 64)];
      const float A2 = fmaf(d[f], d[f], other * other);
      if (mode == FM_SIM) {
        if (ri == 0) a.I_out[((size_t)j * M + ((f + M / 2) % M)) * M + ((idx + M / 2) % M)] = A2;
        continue;
      }
      const float am = amp_global<IST_T>(a, ((size_t)j * M + f) * M + idx, scale);
      if (mode == FM_ERR) {
        if (ri == 0 && am >= 0.f) {
          const float dd = sqrtf(A2) - am;
          en = fmaf(dd, dd, en);
          ed = fmaf(am, am, ed);
        }
        continue;
      }
      d[f] *= proj_factor(mode, am, A2) * inv;
    }
    if (mode == FM_ERR) {
      const double sn = block_sum_d<TC64_NT>(en, red);
      const double sd = block_sum_d<TC64_NT>(ed, red);
      if (tid == 0) {
        a.err_part[(size_t)j * err_c] = make_double2(sn, sd);
        for (int cc = 1; cc < err_c; ++cc) a.err_part[(size_t)j * err_c + cc] = make_double2(0.0, 0.0);
      }
    }
    __syncthreads();  // exchange reads done: the buffer becomes the B tile again
    if (!inverse) continue;
    // ---- inverse: B = conj(D) column-wise (row idx of B = detector column)
    if (ri) {
#pragma unroll
      for (int f = 0; f < 64; ++f) d[f] = -d[f];
    }
#pragma unroll
    for (int g = 0; g < 8; ++g) put8(Bst, idx, 64 * ri + 8 * g, d + 8 * g);
    stage(d);  // D3: d[g] = ri part of conj(V[idx][g]), V the column inverse
#pragma unroll
    for (int g = 0; g < 8; ++g) put8(Bst, idx, 64 * ri + 8 * g, d + 8 * g);
    stage(d);  // D4: d[r] = ri part of conj(chi[r][idx])
    if (ri) {
#pragma unroll
      for (int r = 0; r < 64; ++r) d[r] = -d[r];
    }
    // ---- epilogue: thread (ri, q) writes the ri part of row r, column q
    float* xo = reinterpret_cast<float*>(a.X + (size_t)(j - a.xoff) * M * M);
#pragma unroll
    for (int r = 0; r < 64; ++r) {
      const size_t xi = ((size_t)r * M + idx) * 2 + ri;
      if (mode == FM_CHI || mode == FM_CHIP) {
        if (a.x16) __stcs(reinterpret_cast<unsigned short*>(a.X) + (size_t)(j - a.xoff) * M * M * 2 + xi,
                          __half_as_ushort(__float2half_rn(d[r])));
        else __stcs(xo + xi, d[r]);
      } else {
        const float2 o = __ldg(a.O + (size_t)(p.x + r) * a.nx + p.y + idx);
        const float2 pr = __ldg(Pj + (size_t)r * M + idx);
        __stcs(xo + xi, cpart(cmul(pr, o), ri) + d[r]);
      }
    }
  }
  if (!ok && tid == 0) atomicExch(a.err_flag, 1);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, 64);
}

}  // namespace ptycho

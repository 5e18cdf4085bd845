// Complex helpers and in-register small DFTs (radix 2, 4, 8, 16).
//
// Forward transforms use the kernel exp(-2 pi i n k / N) (numpy fft2
// convention, unnormalised); INV = true uses exp(+2 pi i n k / N).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ptycho {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// conj(a) * b
__device__ __forceinline__ float2 cconjmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.x, b.y, -a.y * b.x));
}
// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialization may become resident while its predecessor in the stream still
// runs; pdl_wait() returns once the predecessor has completed and its writes
// are visible (at once for an ordinary launch: the stream already ordered it),
// pdl_launch() lets the successor start its launch.  Kernels call pdl_wait()
// before their first global access that a predecessor may have written or
// may still read, so either launch form gives stream order.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Bulk prefetch of a contiguous byte range into L2 (the TMA engine issues
// the reads; 16-byte aligned start and size).
__device__ __forceinline__ void prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }

// multiply by -i (forward) or +i (inverse)
template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {
  return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// multiply by (c, -s) forward or (c, s) inverse, i.e. exp(-/+ i theta)
template <bool INV>
__device__ __forceinline__ float2 rot(float2 a, float c, float s) {
  return INV ? make_float2(a.x * c - a.y * s, a.x * s + a.y * c)
             : make_float2(a.x * c + a.y * s, a.y * c - a.x * s);
}

// cos(pi/8), sin(pi/8), sqrt(1/2)
#define PT_C8 0.92387953251128675613f
#define PT_S8 0.38268343236508977173f
#define PT_R2 0.70710678118654752440f

template <bool INV>
__device__ __forceinline__ void dft2(float2* a) {
  float2 t = a[0];
  a[0] = cadd(t, a[1]);
  a[1] = csub(t, a[1]);
}

// a[0..3] with element stride S (in-place, natural order out)
template <bool INV, int S = 1>
__device__ __forceinline__ void dft4s(float2* a) {
  float2 t0 = cadd(a[0], a[2 * S]), t1 = csub(a[0], a[2 * S]);
  float2 t2 = cadd(a[S], a[3 * S]), t3 = mul_mi<INV>(csub(a[S], a[3 * S]));
  a[0] = cadd(t0, t2);
  a[2 * S] = csub(t0, t2);
  a[S] = cadd(t1, t3);
  a[3 * S] = csub(t1, t3);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2* a) { dft4s<INV, 1>(a); }

template <bool INV>
__device__ __forceinline__ void dft8(float2* a) {
  float2 e[4] = {a[0], a[2], a[4], a[6]};
  float2 o[4] = {a[1], a[3], a[5], a[7]};
  dft4<INV>(e);
  dft4<INV>(o);
  o[1] = rot<INV>(o[1], PT_R2, PT_R2);
  o[2] = mul_mi<INV>(o[2]);
  o[3] = rot<INV>(o[3], -PT_R2, PT_R2);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    a[k] = cadd(e[k], o[k]);
    a[k + 4] = csub(e[k], o[k]);
  }
}

// 16-point DFT as 4 x 4 (n = 4 n1 + n2, k = k1 + 4 k2), in place with only
// the temporaries of one radix-4 butterfly live at a time.
template <bool INV>
__device__ __forceinline__ void dft16(float2* a) {
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) dft4s<INV, 4>(a + n2);  // a[n2 + 4 k1] = Y_n2[k1]
  // twiddles W16^(n2 k1)
  a[1 + 4 * 1] = rot<INV>(a[1 + 4 * 1], PT_C8, PT_S8);
  a[1 + 4 * 2] = rot<INV>(a[1 + 4 * 2], PT_R2, PT_R2);
  a[1 + 4 * 3] = rot<INV>(a[1 + 4 * 3], PT_S8, PT_C8);
  a[2 + 4 * 1] = rot<INV>(a[2 + 4 * 1], PT_R2, PT_R2);
  a[2 + 4 * 2] = mul_mi<INV>(a[2 + 4 * 2]);
  a[2 + 4 * 3] = rot<INV>(a[2 + 4 * 3], -PT_R2, PT_R2);
  a[3 + 4 * 1] = rot<INV>(a[3 + 4 * 1], PT_S8, PT_C8);
  a[3 + 4 * 2] = rot<INV>(a[3 + 4 * 2], -PT_R2, PT_R2);
  a[3 + 4 * 3] = rot<INV>(a[3 + 4 * 3], -PT_C8, -PT_S8);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) dft4s<INV, 1>(a + 4 * k1);  // a[4 k1 + k2] = X[k1 + 4 k2]
  // natural order: a 4 x 4 transpose of the register array (renaming only)
  float2 t[16];
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) t[k1 + 4 * k2] = a[4 * k1 + k2];
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i] = t[i];
}


// 3-point DFT: X1,2 = a0 - (a1 + a2)/2 -/+ i (sqrt 3 / 2)(a1 - a2) (forward).
template <bool INV>
__device__ __forceinline__ void dft3(float2* a) {
  const float2 t1 = cadd(a[1], a[2]);
  const float2 m = make_float2(fmaf(-0.5f, t1.x, a[0].x), fmaf(-0.5f, t1.y, a[0].y));
  const float2 d = cscale(csub(a[1], a[2]), 0.86602540378443864676f);
  a[0] = cadd(a[0], t1);
  a[1] = cadd(m, mul_mi<INV>(d));
  a[2] = csub(m, mul_mi<INV>(d));
}

// (cos, sin) of 2 pi e / 24 for e = 1..14
__device__ __constant__ const float2 kTw24[14] = {
  {0.96592582628906831221f, 0.25881904510252073948f},  // e = 1
  {0.86602540378443870761f, 0.49999999999999994449f},  // e = 2
  {0.70710678118654757274f, 0.70710678118654746172f},  // e = 3
  {0.50000000000000011102f, 0.86602540378443859659f},  // e = 4
  {0.25881904510252073948f, 0.96592582628906831221f},  // e = 5
  {0.00000000000000006123f, 1.00000000000000000000f},  // e = 6
  {-0.25881904510252062845f, 0.96592582628906831221f},  // e = 7
  {-0.49999999999999977796f, 0.86602540378443870761f},  // e = 8
  {-0.70710678118654746172f, 0.70710678118654757274f},  // e = 9
  {-0.86602540378443870761f, 0.49999999999999994449f},  // e = 10
  {-0.96592582628906820119f, 0.25881904510252101703f},  // e = 11
  {-1.00000000000000000000f, 0.00000000000000012246f},  // e = 12
  {-0.96592582628906831221f, -0.25881904510252079499f},  // e = 13
  {-0.86602540378443881863f, -0.49999999999999972244f},  // e = 14
};

// 24-point DFT as 8 x 3 (n = 3 n1 + n2, k = k1 + 8 k2).
template <bool INV>
__device__ __forceinline__ void dft24(float2* a) {
#pragma unroll
  for (int n2 = 0; n2 < 3; ++n2) {
    float2 t[8];
#pragma unroll
    for (int n1 = 0; n1 < 8; ++n1) t[n1] = a[3 * n1 + n2];
    dft8<INV>(t);
#pragma unroll
    for (int k1 = 0; k1 < 8; ++k1) {
      float2 v = t[k1];
      const int e = n2 * k1;
      if (e > 0) v = rot<INV>(v, kTw24[e - 1].x, kTw24[e - 1].y);
      a[3 * k1 + n2] = v;  // Y[n2][k1]
    }
  }
#pragma unroll
  for (int k1 = 0; k1 < 8; ++k1) dft3<INV>(a + 3 * k1);  // a[3 k1 + k2] = X[k1 + 8 k2]
  float2 t[24];
#pragma unroll
  for (int k1 = 0; k1 < 8; ++k1)
#pragma unroll
    for (int k2 = 0; k2 < 3; ++k2) t[k1 + 8 * k2] = a[3 * k1 + k2];
#pragma unroll
  for (int i = 0; i < 24; ++i) a[i] = t[i];
}

template <int R, bool INV>
__device__ __forceinline__ void dft(float2* a) {
  if constexpr (R == 2) dft2<INV>(a);
  else if constexpr (R == 4) dft4<INV>(a);
  else if constexpr (R == 8) dft8<INV>(a);
  else if constexpr (R == 16) dft16<INV>(a);
  else if constexpr (R == 3) dft3<INV>(a);
  else if constexpr (R == 24) dft24<INV>(a);
  else static_assert(R == 2 || R == 4 || R == 8 || R == 16 || R == 3 || R == 24, "radix");
}

// Radix of the next Stockham pass for a remaining length rem, given that a
// thread holds E elements (the radix must divide E).
__host__ __device__ constexpr int pick_radix(int rem, int E) {
  int cap = E < 16 ? E : 16;
  if (rem <= cap) return rem;
  if (rem == 32 && cap >= 8) return 8;        // 8 x 4
  if (rem == 64 && cap >= 8) return 8;        // 8 x 8
  return cap;
}

// ---------------------------------------------------------------------------
// One Stockham autosort pass of radix R over LINES lines of length N held in
// shared memory (Stockham's self-sorting variant of Cooley-Tukey: every pass
// reads with stride N/R and writes in natural order, so no bit reversal is
// needed).  NS = product of the radices of the earlier passes.
//
// Element i of line l lives at  (l / LPB) * BS + (l % LPB) * LS + i * IS.
// The NT threads each take PER butterflies (b = tid + p*NT, line = b % LINES,
// so a warp spans consecutive lines), load them all into registers, sync,
// then store, which makes the pass in place.
// tw[i] = exp(-2 pi i i / N) for i < N (table of the line length).
// ---------------------------------------------------------------------------
template <int N, int R, int NS, int LINES, int LPB, int BS, int LS, int IS, int NT, bool INV>
__device__ __forceinline__ void stockham_pass(float2* s, const float2* __restrict__ tw) {
  constexpr int BPL = N / R;
  constexpr int TOT = LINES * BPL;
  constexpr int PER = (TOT + NT - 1) / NT;
  constexpr int TWS = N / (NS * R);
  float2 v[PER][R];
  const int tid = threadIdx.x;
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int b = tid + p * NT;
    if (TOT % NT == 0 || b < TOT) {
      const int l = b % LINES, jj = b / LINES;
      const int base = (l / LPB) * BS + (l % LPB) * LS;
#pragma unroll
      for (int r = 0; r < R; ++r) v[p][r] = s[base + (jj + r * BPL) * IS];
      if constexpr (NS > 1) {
        const int jm = jj % NS;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          float2 w = tw[(r * jm * TWS) % N];
          if (INV) w.y = -w.y;
          v[p][r] = cmul(v[p][r], w);
        }
      }
      dft<R, INV>(v[p]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int b = tid + p * NT;
    if (TOT % NT == 0 || b < TOT) {
      const int l = b % LINES, jj = b / LINES;
      const int base = (l / LPB) * BS + (l % LPB) * LS;
      const int jm = jj % NS;
      const int d = (jj / NS) * NS * R + jm;
#pragma unroll
      for (int r = 0; r < R; ++r) s[base + (d + r * NS) * IS] = v[p][r];
    }
  }
  __syncthreads();
}

// Full length-N FFT of every line: the sequence of passes chosen by pick_radix.
template <int N, int NS, int E, int LINES, int LPB, int BS, int LS, int IS, int NT, bool INV>
__device__ __forceinline__ void fft_lines_from(float2* s, const float2* __restrict__ tw) {
  if constexpr (NS < N) {
    constexpr int R = pick_radix(N / NS, E);
    stockham_pass<N, R, NS, LINES, LPB, BS, LS, IS, NT, INV>(s, tw);
    fft_lines_from<N, NS * R, E, LINES, LPB, BS, LS, IS, NT, INV>(s, tw);
  }
}

template <int N, int E, int LINES, int LPB, int BS, int LS, int IS, int NT, bool INV>
__device__ __forceinline__ void fft_lines(float2* s, const float2* __restrict__ tw) {
  fft_lines_from<N, 1, E, LINES, LPB, BS, LS, IS, NT, INV>(s, tw);
}

// Block-wide sum of doubles (any NT <= 1024); result valid in thread 0.
template <int NT>
__device__ __forceinline__ double block_sum_d(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  constexpr int NW = (NT + 31) / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < NW; ++i) t += red[i];
  }
  return t;
}

template <int NT>
__device__ __forceinline__ float block_max_f(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
  constexpr int NW = (NT + 31) / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x == 0) {
    for (int i = 0; i < NW; ++i) t = fmaxf(t, red[i]);
  }
  return t;
}

}  // namespace ptycho

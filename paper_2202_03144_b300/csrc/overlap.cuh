// Overlap accumulation of the DM / LSQML object and probe updates.
//
// Object side (tile-owned, atomic-free, deterministic): each CTA owns a
// TY x TX tile of the object and walks, in ascending position order, the CSR
// list of scan positions whose patch overlaps the tile.  Every thread owns
// fixed pixels and accumulates in registers
//     num(r) = sum_j w_j sum_k conj(P_k(r - p_j)) X_jk(r - p_j)
//     den(r) = sum_j sum_k |P_k(r - p_j)|^2
// so each element of X (psi or chi) is read exactly once overall and a warp
// reads 32 consecutive complex values of one patch row.
//
// Probe side: num_P,k(u) = sum_j w_j conj(O_j(u)) X_jk(u), den_P(u) = sum_j
// |O_j(u)|^2.  The positions are cut into G contiguous groups; CTA (block,
// group) sums its group for 256 probe pixels, and a second kernel adds the G
// partials in a fixed order.
//
// Sub-pixel positions: P is a table of shifted probes, [bins][K][M][M], and
// position j reads bin pbin[j]; on the probe side the positions are taken in
// bin order and the groups never straddle a bin, so the fixed-order sum
// yields one numerator per bin (the caller then applies the adjoint shifts).
#pragma once
#include <cuda_fp16.h>

#include "common.cuh"

namespace ptycho {

constexpr int TILE_Y = 32, TILE_X = 64, OBJ_NT = 256;
// A thread owns OBJ_COLS adjacent columns of OBJ_ROWS rows of its tile: the
// index arithmetic and bounds tests of a (position, row) step are shared by
// four pixels, and the loads are 16 bytes wide when the patch column offset
// is even (the pixel pairs are then aligned and never straddle the patch edge).
constexpr int OBJ_COLS = 4;
constexpr int OBJ_TX = TILE_X / OBJ_COLS;              // threads across the tile (16)
constexpr int OBJ_RSTEP = OBJ_NT / OBJ_TX;             // row stride between a thread's rows (16)
constexpr int OBJ_ROWS = TILE_Y / OBJ_RSTEP;           // rows per thread (2)
constexpr int PROBE_NT = 256;
#ifndef PT_OBJ_MINB
#define PT_OBJ_MINB 4     // occupancy hint (CTAs per SM) of the object kernel (4: 1.06 ms vs 1.12 at 3)
#endif
// Step-size kernel: one pixel pair per thread per step at 4 CTAs per SM
// measured fastest (3.9 TB/s against 3.6 for two pairs at the default
// occupancy); it also reads ~40 B/pixel from L2 (O, dO, P, dP) per 8 B of chi.
#ifndef PT_STEP_PF
#define PT_STEP_PF 4      // residual L2 prefetch distance of the step-size kernel, in loop steps (0: none)
#endif
#ifndef PT_STEP_MINB
#define PT_STEP_MINB 4    // occupancy hint of the LSQML step-size kernel
#endif
#ifndef PT_PROBE_UJ
#define PT_PROBE_UJ 8     // positions per step of the probe sums, K = 1 (8: 0.945 ms vs 1.03 at 4, 1.22 at 16)
#endif
#ifndef PT_PROBE_UJ16
#define PT_PROBE_UJ16 4   // the same for FP16 residuals (two pixels per thread)
#endif
#ifndef PT_STEP_UNROLL
#define PT_STEP_UNROLL 1  // pixel-loop unrolling of the step-size kernel
#endif
#define PT_PRAGMA(x) _Pragma(#x)
#define PT_UNROLL(n) PT_PRAGMA(unroll n)
// Residual loads: X holds FP32 complex values (float2) or, with FP16
// residual storage, __half2; either way the kernels compute in FP32.
// ld_x: element i; ld_x2: elements i and i + 1 (i even) as one float4.
template <typename XT>
__device__ __forceinline__ float2 ld_x(const float2* X, size_t i) {
  if constexpr (sizeof(XT) == 8) return __ldcs(X + i);
  else return __half22float2(__ldcs(reinterpret_cast<const __half2*>(X) + i));
}
template <typename XT>
__device__ __forceinline__ float4 ld_x2(const float2* X, size_t i) {
  if constexpr (sizeof(XT) == 8) {
    return __ldcs(reinterpret_cast<const float4*>(X + i));
  } else {
    const uint2 u = __ldcs(reinterpret_cast<const uint2*>(reinterpret_cast<const __half2*>(X) + i));
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
    return make_float4(a.x, a.y, b.x, b.y);
  }
}

constexpr int OBJ_CHUNK = 256;   // positions staged per chunk (k_obj)
constexpr int PROBE_CHUNK = 512; // positions staged per chunk (k_probe_partial)

// OBJ_NUMDEN: numerator (unweighted, to dO) and den_O (to den) in one pass,
//             with the per-tile maximum of den_O; k_obj_norm then applies the
//             DM update or forms the LSQML direction.
// OBJ_UPD:    LSQML update O += beta sum_j alpha_j S_j[...] / (den_O + delta).
enum ObjMode : int { OBJ_NUMDEN = 0, OBJ_UPD = 3 };
enum NormMode : int { NORM_DM = 0, NORM_DIR = 1 };
enum ProbeMode : int { PR_DM = 0, PR_DIR = 1, PR_UPD = 2 };

struct ObjArgs {
  float2* O;              // object (DM, UPD: in/out)
  float2* dO;             // DIR: output direction
  int ny, nx, ntx;        // object size, tiles per row
  const float2* P;        // probe [K][M][M], or the shifted table [bins][K][M][M]
  const unsigned short* pbin;  // sub-pixel bin of each position, or NULL
  const float2* X;        // psi or chi [J][K][M][M]
  const int2* pos;
  const int* tile_ptr;    // [n_tiles + 1]
  const int* tile_list;   // positions overlapping each tile, ascending
  const float* weights;   // per-position weight (alpha_O) or NULL
  float* den;             // den_O [ny][nx] (written by OBJ_NUMDEN, read otherwise);
                          // OBJ_NUMDEN with NULL: numerator only
  float* tile_max;        // OBJ_NUMDEN: max of den per tile
  const float* den_max;   // max over all tiles (one float)
  float reg, beta;
  int M;
  // position blocks (residuals of positions [jlo, jhi) only, X holding
  // them from position xoff on); accumulate: OBJ_NUMDEN adds to dO / den
  int jlo, jhi, xoff, accumulate;
};

// SUB: sub-pixel positions (P is the shifted table, indexed by pbin).
template <int K, int MODE, bool SUB, typename XT = float2>
__global__ void __launch_bounds__(OBJ_NT, K == 1 ? PT_OBJ_MINB : 3) k_obj(ObjArgs a) {  // K > 1: 3 (no spills)
  __shared__ float red[32];
  const int tile = blockIdx.x;
  const int ty0 = (tile / a.ntx) * TILE_Y, tx0 = (tile % a.ntx) * TILE_X;
  const int cx = threadIdx.x % OBJ_TX, ry = threadIdx.x / OBJ_TX;
  const int x = tx0 + OBJ_COLS * cx;  // first of this thread's columns (even)
  const int M = a.M;
  const size_t MM = (size_t)M * M;
  float2 num[OBJ_ROWS][OBJ_COLS];
  float den[OBJ_ROWS][OBJ_COLS];
#pragma unroll
  for (int i = 0; i < OBJ_ROWS; ++i)
#pragma unroll
    for (int e = 0; e < OBJ_COLS; ++e) {
      num[i][e] = make_float2(0.f, 0.f);
      den[i][e] = 0.f;
    }
  int s0 = a.tile_ptr[tile], s1 = a.tile_ptr[tile + 1];
  if (a.jhi > a.jlo) {  // a block of positions: the tile's list is ascending, cut it by bisection
    int lo = s0, hi = s1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (a.tile_list[mid] < a.jlo) lo = mid + 1; else hi = mid;
    }
    const int b0 = lo;
    hi = s1;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (a.tile_list[mid] < a.jhi) lo = mid + 1; else hi = mid;
    }
    s0 = b0;
    s1 = lo;
  }
  // the tile's positions (index, corner, weight) staged in shared memory in
  // chunks, so the inner loop has no chain of dependent global loads
  __shared__ int sj[OBJ_CHUNK];
  __shared__ int2 sp[OBJ_CHUNK];
  __shared__ float sw[OBJ_CHUNK];
  __shared__ int sb[SUB ? OBJ_CHUNK : 1];
  const bool weighted = a.weights != nullptr;
  for (int c0 = s0; c0 < s1; c0 += OBJ_CHUNK) {
    const int nc = min(OBJ_CHUNK, s1 - c0);
    __syncthreads();
    for (int i = threadIdx.x; i < nc; i += OBJ_NT) {
      const int j = a.tile_list[c0 + i];
      sj[i] = j;
      sp[i] = a.pos[j];
      sw[i] = weighted ? a.weights[j] : 1.f;
      if (SUB) sb[i] = a.pbin[j];
    }
    __syncthreads();
    for (int s = 0; s < nc; ++s) {
      const int j = sj[s];
      const int2 p = sp[s];
      const float w = sw[s];
      const float2* Pj = SUB ? a.P + (size_t)sb[s] * K * MM : a.P;
      const int ux = x - p.y;                 // patch column of this thread's first pixel
      const bool pairs = ((ux & 1) == 0);     // uniform over the CTA (x is even)
      // one mode at a time (the per-pixel order of the sums is unchanged)
#pragma unroll
      for (int k = 0; k < K; ++k) {
        float2 pv[OBJ_ROWS][OBJ_COLS], xv[OBJ_ROWS][OBJ_COLS];
#pragma unroll
        for (int i = 0; i < OBJ_ROWS; ++i) {
          const int uy = ty0 + ry + OBJ_RSTEP * i - p.x;
          const bool row_in = uy >= 0 && uy < M;
          const size_t u0 = (size_t)(row_in ? uy : 0) * M;
          const float2* prow = Pj + k * MM + u0;
          const size_t xrow = ((size_t)(j - a.xoff) * K + k) * MM + u0;  // element index in X
          if (pairs) {
#pragma unroll
            for (int e = 0; e < OBJ_COLS; e += 2) {
              const bool in = row_in && ux + e >= 0 && ux + e < M;  // both pixels of the pair
              float4 pq = make_float4(0.f, 0.f, 0.f, 0.f), xq = pq;
              if (in) {
                pq = __ldg(reinterpret_cast<const float4*>(prow + ux + e));
                xq = ld_x2<XT>(a.X, xrow + ux + e);
              }
              pv[i][e] = make_float2(pq.x, pq.y);
              pv[i][e + 1] = make_float2(pq.z, pq.w);
              xv[i][e] = make_float2(xq.x, xq.y);
              xv[i][e + 1] = make_float2(xq.z, xq.w);
            }
          } else {
#pragma unroll
            for (int e = 0; e < OBJ_COLS; ++e) {
              const bool in = row_in && ux + e >= 0 && ux + e < M;
              pv[i][e] = in ? __ldg(prow + ux + e) : make_float2(0.f, 0.f);
              xv[i][e] = in ? ld_x<XT>(a.X, xrow + ux + e) : make_float2(0.f, 0.f);
            }
          }
        }
#pragma unroll
        for (int i = 0; i < OBJ_ROWS; ++i)
#pragma unroll
          for (int e = 0; e < OBJ_COLS; ++e) {
            if (MODE == OBJ_NUMDEN) den[i][e] += cabs2(pv[i][e]);
            const float2 t = cconjmul(pv[i][e], xv[i][e]);
            num[i][e].x = fmaf(w, t.x, num[i][e].x);
            num[i][e].y = fmaf(w, t.y, num[i][e].y);
          }
      }
    }
  }
  if (MODE == OBJ_NUMDEN) {
    float m = 0.f;
    const bool want_den = a.den != nullptr;
#pragma unroll
    for (int i = 0; i < OBJ_ROWS; ++i)
#pragma unroll
      for (int e = 0; e < OBJ_COLS; ++e) {
        const int y = ty0 + ry + OBJ_RSTEP * i;
        if (y < a.ny && x + e < a.nx) {
          const size_t r = (size_t)y * a.nx + x + e;
          float d = den[i][e];
          float2 nm = num[i][e];
          if (a.accumulate) {
            nm = cadd(a.dO[r], nm);
            if (want_den) d += a.den[r];
          }
          if (want_den) a.den[r] = d;
          a.dO[r] = nm;
          m = fmaxf(m, d);
        }
      }
    if (!want_den) return;
    m = block_max_f<OBJ_NT>(m, red);
    if (threadIdx.x == 0) a.tile_max[tile] = m;
    return;
  }
  const float delta = a.reg * a.den_max[0];
#pragma unroll
  for (int i = 0; i < OBJ_ROWS; ++i)
#pragma unroll
    for (int e = 0; e < OBJ_COLS; ++e) {
      const int y = ty0 + ry + OBJ_RSTEP * i;
      if (y >= a.ny || x + e >= a.nx) continue;
      const size_t r = (size_t)y * a.nx + x + e;
      const float d = a.den[r] + delta;
      const float inv = d > 0.f ? 1.f / d : 0.f;
      const float2 o = a.O[r];
      const float sc = a.beta * inv;
      a.O[r] = make_float2(fmaf(sc, num[i][e].x, o.x), fmaf(sc, num[i][e].y, o.y));
    }
}

// Object-sized epilogue of OBJ_NUMDEN, with delta = reg * max(den_O):
//   NORM_DM:  O  <- (num + delta O) / (den + delta)
//   NORM_DIR: dO <- num / (den + delta)          (num is held in dO)
template <int MODE>
__global__ void __launch_bounds__(256) k_obj_norm(float2* __restrict__ O, float2* __restrict__ dO,
                                                  const float* __restrict__ den, const float* __restrict__ den_max,
                                                  float reg, size_t n) {
  const float delta = reg * den_max[0];
  for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r < n; r += (size_t)gridDim.x * blockDim.x) {
    const float d = den[r] + delta;
    const float inv = d > 0.f ? 1.f / d : 0.f;
    const float2 num = dO[r];
    if (MODE == NORM_DM) {
      const float2 o = O[r];
      O[r] = make_float2(fmaf(delta, o.x, num.x) * inv, fmaf(delta, o.y, num.y) * inv);
    } else {
      dO[r] = cscale(num, inv);
    }
  }
}

// LSQML update from an accumulated numerator (position blocks):
//   O <- O + beta acc / (den + delta)
__global__ void __launch_bounds__(256) k_obj_apply_acc(float2* __restrict__ O, const float2* __restrict__ acc,
                                                       const float* __restrict__ den, const float* __restrict__ den_max,
                                                       float reg, float beta, size_t n) {
  const float delta = reg * den_max[0];
  for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r < n; r += (size_t)gridDim.x * blockDim.x) {
    const float d = den[r] + delta;
    const float sc = beta * (d > 0.f ? 1.f / d : 0.f);
    const float2 o = O[r], num = acc[r];
    O[r] = make_float2(fmaf(sc, num.x, o.x), fmaf(sc, num.y, o.y));
  }
}

// Max of n floats into out[0] (one CTA, fixed order).
__global__ void __launch_bounds__(1024) k_reduce_max(const float* in, int n, float* out) {
  __shared__ float red[32];
  float m = 0.f;
  for (int i = threadIdx.x; i < n; i += 1024) m = fmaxf(m, in[i]);
  m = block_max_f<1024>(m, red);
  if (threadIdx.x == 0) out[0] = m;
}

struct ProbeArgs {
  const float2* O;
  int nx;
  const float2* X;         // [J][K][M][M]
  const int2* pos;
  const float* weights;    // alpha_P or NULL
  const int* order;        // positions in group order (sub-pixel: by bin), or NULL = 0..J-1
  const int* goff;         // [G + 1] group offsets into the order, or NULL = even split of J
  const int* bgrp;         // [bins + 1] first group of each bin (sub-pixel), or NULL
  int nbins;
  int J, M, G;
  int jlo, xoff;           // position blocks: positions [jlo, jlo + J), X from position xoff on
  int accumulate;          // k_probe_sum adds to num / den
  float2* part_num;        // [G][K][M*M]
  float* part_den;         // [G][M*M] or NULL (skip den)
  float2* num;             // [K][M*M] (sub-pixel: [bins][K][M*M])
  float* den;              // [M*M]
  float* bin_den;          // sub-pixel: per-bin den [bins][M*M], or NULL
  float* blk_max;          // [ceil(M*M/256)]
  float2* P;               // PR_DM, PR_UPD: in/out
  float2* dP;              // PR_DIR: out
  float reg, beta;
};

// SUB: positions taken through the bin order and its group offsets.
// Pixels per thread: one for FP32 residuals, two adjacent ones (in one row, M
// being even) for FP16 residuals of one mode, whose 4-byte values would
// otherwise halve the bytes each load request moves (with three modes the
// two-pixel form needs over 100 registers).  Each pixel sums its positions
// in the same order either way.
#ifndef PT_PROBE_MINB
#define PT_PROBE_MINB 1   // occupancy hint of the probe partial sums (1: none)
#endif
template <typename XT, int K>
__host__ __device__ constexpr int probe_px() {
  return sizeof(XT) == 4 && K == 1 ? 2 : 1;
}
template <int K, bool SUB, typename XT = float2>
__global__ void __launch_bounds__(PROBE_NT, PT_PROBE_MINB) k_probe_partial(ProbeArgs a) {
  constexpr int PX = probe_px<XT, K>();
  const int MM = a.M * a.M;
  const int u = (blockIdx.x * PROBE_NT + threadIdx.x) * PX;  // first pixel of this thread
  const int uy = u / a.M, ux = u % a.M;
  const int g = blockIdx.y;
  const int jb = SUB ? a.goff[g] : a.jlo + (int)(((long long)a.J * g) / a.G);
  const int je = SUB ? a.goff[g + 1] : a.jlo + (int)(((long long)a.J * (g + 1)) / a.G);
  float2 num[PX][K];
  float den[PX];
#pragma unroll
  for (int e = 0; e < PX; ++e) {
    den[e] = 0.f;
#pragma unroll
    for (int k = 0; k < K; ++k) num[e][k] = make_float2(0.f, 0.f);
  }
  const bool want_den = a.part_den != nullptr;
  // positions per step: UJ*(K+1) independent loads in flight
  constexpr int UJ = PX == 2 ? PT_PROBE_UJ16 : (K == 1 ? PT_PROBE_UJ : 4);
  __shared__ int2 sp[PROBE_CHUNK];
  __shared__ float sw[PROBE_CHUNK];
  __shared__ int sj[SUB ? PROBE_CHUNK : 1];
  for (int c0 = jb; c0 < je; c0 += PROBE_CHUNK) {
    const int nc = min(PROBE_CHUNK, je - c0);
    __syncthreads();
    for (int i = threadIdx.x; i < nc; i += PROBE_NT) {
      const int j = SUB ? a.order[c0 + i] : c0 + i;
      if (SUB) sj[i] = j;
      sp[i] = a.pos[j];
      sw[i] = a.weights ? a.weights[j] : 1.f;
    }
    __syncthreads();
    if (u < MM) {
      for (int s = 0; s < nc; s += UJ) {
        float2 o[UJ][PX], xv[UJ][K][PX];
        float w[UJ];
#pragma unroll
        for (int h = 0; h < UJ; ++h) {
          const bool in = s + h < nc;
          const int i = in ? s + h : 0;
          const int2 p = sp[i];
          if constexpr (PX == 1) {
            o[h][0] = in ? __ldg(a.O + (size_t)(p.x + uy) * a.nx + p.y + ux) : make_float2(0.f, 0.f);
          } else {
            const size_t r = (size_t)(p.x + uy) * a.nx + p.y + ux;
            // the object pixel pair is 16-byte aligned when the patch's first
            // column and the row length are even (uniform over the block)
            float4 oq = make_float4(0.f, 0.f, 0.f, 0.f);
            if (in && ((p.y | a.nx) & 1) == 0) {
              oq = __ldg(reinterpret_cast<const float4*>(a.O + r));
            } else if (in) {
              const float2 o0 = __ldg(a.O + r), o1 = __ldg(a.O + r + 1);
              oq = make_float4(o0.x, o0.y, o1.x, o1.y);
            }
            o[h][0] = make_float2(oq.x, oq.y);
            o[h][1] = make_float2(oq.z, oq.w);
          }
          w[h] = in ? sw[i] : 0.f;
#pragma unroll
          for (int k = 0; k < K; ++k) {
            if constexpr (PX == 1) {
              xv[h][k][0] = in ? ld_x<XT>(a.X, ((size_t)((SUB ? sj[i] : c0 + i) - a.xoff) * K + k) * MM + u)
                               : make_float2(0.f, 0.f);
            } else {
              const size_t xi = ((size_t)((SUB ? sj[i] : c0 + i) - a.xoff) * K + k) * MM + u;
              const float4 xq = in ? ld_x2<XT>(a.X, xi) : make_float4(0.f, 0.f, 0.f, 0.f);
              xv[h][k][0] = make_float2(xq.x, xq.y);
              xv[h][k][1] = make_float2(xq.z, xq.w);
            }
          }
        }
#pragma unroll
        for (int h = 0; h < UJ; ++h)
#pragma unroll
          for (int e = 0; e < PX; ++e) {
            if (want_den) den[e] += cabs2(o[h][e]);
#pragma unroll
            for (int k = 0; k < K; ++k) {
              const float2 t = cconjmul(o[h][e], xv[h][k][e]);
              num[e][k].x = fmaf(w[h], t.x, num[e][k].x);
              num[e][k].y = fmaf(w[h], t.y, num[e][k].y);
            }
          }
      }
    }
  }
  if (u >= MM) return;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    float2* dst = a.part_num + ((size_t)g * K + k) * MM + u;
    if constexpr (PX == 1) *dst = num[0][k];
    else *reinterpret_cast<float4*>(dst) = make_float4(num[0][k].x, num[0][k].y, num[1][k].x, num[1][k].y);
  }
  if (want_den) {
    float* dst = a.part_den + (size_t)g * MM + u;
    if constexpr (PX == 1) *dst = den[0];
    else *reinterpret_cast<float2*>(dst) = make_float2(den[0], den[1]);
  }
}

// Sum the G partials in group order (sub-pixel: per bin, into num[bin]);
// block maxima of den for the regulariser.
template <int K>
__global__ void __launch_bounds__(PROBE_NT) k_probe_sum(ProbeArgs a) {
  __shared__ float red[32];
  const int MM = a.M * a.M;
  const int u = blockIdx.x * PROBE_NT + threadIdx.x;
  const bool want_den = a.part_den != nullptr;
  float m = 0.f;
  if (u < MM) {
    const int nb = a.bgrp ? a.nbins : 1;
    for (int b = 0; b < nb; ++b) {
      const int g0 = a.bgrp ? a.bgrp[b] : 0, g1 = a.bgrp ? a.bgrp[b + 1] : a.G;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        float2 s = make_float2(0.f, 0.f);
        for (int g = g0; g < g1; ++g) s = cadd(s, a.part_num[((size_t)g * K + k) * MM + u]);
        const size_t o = ((size_t)b * K + k) * MM + u;
        a.num[o] = a.accumulate ? cadd(a.num[o], s) : s;
      }
    }
    if (want_den) {
      float d = 0.f;
      for (int g = 0; g < a.G; ++g) d += a.part_den[(size_t)g * MM + u];
      if (a.accumulate) d += a.den[u];
      a.den[u] = d;
      m = d;
      if (a.bgrp && a.bin_den)
        for (int b = 0; b < a.nbins; ++b) {
          float db = 0.f;
          for (int g = a.bgrp[b]; g < a.bgrp[b + 1]; ++g) db += a.part_den[(size_t)g * MM + u];
          a.bin_den[(size_t)b * MM + u] = db;
        }
    }
  }
  if (want_den) {
    m = block_max_f<PROBE_NT>(m, red);
    if (threadIdx.x == 0) a.blk_max[blockIdx.x] = m;
  }
}

template <int K, int MODE>
__global__ void __launch_bounds__(PROBE_NT) k_probe_apply(ProbeArgs a) {
  __shared__ float red[32];
  __shared__ float s_max;
  const int MM = a.M * a.M;
  const int nblk = (MM + PROBE_NT - 1) / PROBE_NT;
  float m = 0.f;
  for (int i = threadIdx.x; i < nblk; i += PROBE_NT) m = fmaxf(m, a.blk_max[i]);
  m = block_max_f<PROBE_NT>(m, red);
  if (threadIdx.x == 0) s_max = m;
  __syncthreads();
  const int u = blockIdx.x * PROBE_NT + threadIdx.x;
  if (u >= MM) return;
  const float delta = a.reg * s_max;
  const float d = a.den[u] + delta;
  const float inv = d > 0.f ? 1.f / d : 0.f;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const size_t i = (size_t)k * MM + u;
    const float2 n = a.num[i];
    if (MODE == PR_DM) {
      const float2 pr = a.P[i];
      a.P[i] = make_float2(fmaf(delta, pr.x, n.x) * inv, fmaf(delta, pr.y, n.y) * inv);
    } else if (MODE == PR_DIR) {
      a.dP[i] = cscale(n, inv);
    } else {
      const float2 pr = a.P[i];
      const float sc = a.beta * inv;
      a.P[i] = make_float2(fmaf(sc, n.x, pr.x), fmaf(sc, n.y, pr.y));
    }
  }
}

// ---------------------------------------------------------------------------
// LSQML per-position step sizes.  a_k = P_k dO_j, b_k = O_j dP_k; the five
// sums |a|^2, Re<a,b>, |b|^2, Re<a,chi>, Re<b,chi> are accumulated per thread
// in FP32 and across the block in FP64; the regularised 2x2 system
// (lambda = 1e-6 (A11 + A22) / 2) is solved in FP64 by one thread.
// ---------------------------------------------------------------------------
struct StepArgs {
  const float2* O;
  const float2* dO;
  int nx;
  const float2* P;    // probe, or the shifted table [bins][K][M][M]
  const float2* dP;   // NULL when the probe is fixed (sub-pixel: shifted table)
  const unsigned short* pbin;  // sub-pixel bin of each position, or NULL
  const float2* X;    // chi
  const int2* pos;
  int M;
  float* alpha_O;
  float* alpha_P;
  int j0, xoff;       // first position of the launch; X holds positions from xoff on
  int nj;             // positions of the launch
};

constexpr int STEP_NT = 256;

// SUB: sub-pixel positions (P and dP are shifted tables indexed by pbin); the
// extra offset costs registers, so K = 3 then runs at three CTAs per SM.
template <int K, bool SUB, typename XT = float2>
__global__ void __launch_bounds__(STEP_NT, (SUB && K == 3) ? 3 : PT_STEP_MINB) k_lsqml_steps(StepArgs a) {
  __shared__ double red[32];
  const int j = a.j0 + blockIdx.x;
  const int2 p = a.pos[j];
  const int MM = a.M * a.M;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, s4 = 0.f;
  const bool upd = a.dP != nullptr;
  const size_t boff = SUB ? (size_t)a.pbin[j] * K * MM : 0;  // sub-pixel: this position's table bin
  // two adjacent pixels per thread (16-byte loads of chi, P, dP; M is even so
  // both lie in one row); the pixel's row and column advance incrementally
  const int M = a.M;
  constexpr int STEP = 2 * STEP_NT;
  const int dy = STEP / M, dx = STEP % M;
  int u = 2 * threadIdx.x;
  int uy = u / M, ux = u % M;
  // the object pixel pair is 16-byte aligned when the patch's first object
  // column and the row length are even (uniform over the block)
  const bool pairs = ((p.y | a.nx) & 1) == 0;
  // this position's residuals, streamed from HBM: thread 0 keeps the next
  // PT_STEP_PF loop steps' chunks (STEP values per mode) on their way to L2
  const size_t xj = (size_t)(j - a.xoff) * K * MM;  // element index of this position's residuals
  const unsigned char* xb = reinterpret_cast<const unsigned char*>(a.X);
  if (PT_STEP_PF > 0 && threadIdx.x == 0)
    for (int q = 0; q < PT_STEP_PF && q * STEP < MM; ++q)
#pragma unroll
      for (int k = 0; k < K; ++k)
        prefetch_l2(xb + (xj + (size_t)k * MM + q * STEP) * sizeof(XT), (uint32_t)(min(STEP, MM - q * STEP) * sizeof(XT)));
  PT_UNROLL(PT_STEP_UNROLL)
  for (; u < MM; u += STEP) {
    if (PT_STEP_PF > 0 && threadIdx.x == 0) {
      const int ua = u + PT_STEP_PF * STEP;   // thread 0's u is the step's first value
      if (ua < MM)
#pragma unroll
        for (int k = 0; k < K; ++k)
          prefetch_l2(xb + (xj + (size_t)k * MM + ua) * sizeof(XT), (uint32_t)(min(STEP, MM - ua) * sizeof(XT)));
    }
    const size_t r = (size_t)(p.x + uy) * a.nx + p.y + ux;
    float2 o0, o1, d0, d1;
    if (pairs) {
      const float4 oq = __ldg(reinterpret_cast<const float4*>(a.O + r));
      const float4 dq = __ldg(reinterpret_cast<const float4*>(a.dO + r));
      o0 = make_float2(oq.x, oq.y), o1 = make_float2(oq.z, oq.w);
      d0 = make_float2(dq.x, dq.y), d1 = make_float2(dq.z, dq.w);
    } else {
      o0 = __ldg(a.O + r), o1 = __ldg(a.O + r + 1);
      d0 = __ldg(a.dO + r), d1 = __ldg(a.dO + r + 1);
    }
    float4 xv[K], pr[K], dp[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      pr[k] = __ldg(reinterpret_cast<const float4*>(a.P + boff + (size_t)k * MM + u));
      xv[k] = ld_x2<XT>(a.X, xj + (size_t)k * MM + u);
      dp[k] = upd ? __ldg(reinterpret_cast<const float4*>(a.dP + boff + (size_t)k * MM + u)) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const float2 oo = e ? o1 : o0;
      const float2 dd = e ? d1 : d0;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float2 pk = e ? make_float2(pr[k].z, pr[k].w) : make_float2(pr[k].x, pr[k].y);
        const float2 xk = e ? make_float2(xv[k].z, xv[k].w) : make_float2(xv[k].x, xv[k].y);
        const float2 av = cmul(pk, dd);
        s0 += cabs2(av);
        s3 += fmaf(av.x, xk.x, av.y * xk.y);
        if (upd) {
          const float2 dk = e ? make_float2(dp[k].z, dp[k].w) : make_float2(dp[k].x, dp[k].y);
          const float2 bv = cmul(oo, dk);
          s1 += fmaf(av.x, bv.x, av.y * bv.y);
          s2 += cabs2(bv);
          s4 += fmaf(bv.x, xk.x, bv.y * xk.y);
        }
      }
    }
    ux += dx;
    uy += dy;
    if (ux >= M) {
      ux -= M;
      ++uy;
    }
  }
  const double A11 = block_sum_d<STEP_NT>(s0, red);
  const double A12 = block_sum_d<STEP_NT>(s1, red);
  const double A22 = block_sum_d<STEP_NT>(s2, red);
  const double r1 = block_sum_d<STEP_NT>(s3, red);
  const double r2 = block_sum_d<STEP_NT>(s4, red);
  if (threadIdx.x == 0) {
    double aO = 0.0, aP = 0.0;
    const double tr = A11 + A22;
    if (tr > 0.0) {
      const double lam = 1e-6 * tr / 2.0;
      const double a11 = A11 + lam, a22 = A22 + lam;
      const double det = a11 * a22 - A12 * A12;
      aO = (a22 * r1 - A12 * r2) / det;
      aP = (a11 * r2 - A12 * r1) / det;
    }
    a.alpha_O[j] = (float)aO;
    a.alpha_P[j] = (float)aP;
  }
}

// ---------------------------------------------------------------------------
// Position correction (sub-pixel positions): per position the shift s that
// best explains the residual, a_y = P_jk dO/dy, a_x = P_jk dO/dx (central
// differences of the object, an index past the edge clamped to it), sums in
// FP32 per thread and FP64 across the block, the regularised 2x2 system
// solved in FP64 as for the LSQML step sizes.  out[j] = (s_y, s_x).
// ---------------------------------------------------------------------------
struct PosCorrArgs {
  const float2* O;
  int ny, nx;
  const float2* P;             // shifted-probe table [bins][K][M][M]
  const unsigned short* pbin;
  const float2* X;             // chi
  const int2* pos;
  int M;
  float2* out;
};

template <int K>
__global__ void __launch_bounds__(STEP_NT) k_pos_corr(PosCorrArgs a) {
  __shared__ double red[32];
  const int j = blockIdx.x;
  const int2 p = a.pos[j];
  const int M = a.M, MM = M * M;
  const float2* Pj = a.P + (size_t)a.pbin[j] * K * MM;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, s4 = 0.f;
  for (int u = threadIdx.x; u < MM; u += STEP_NT) {
    const int y = p.x + u / M, x = p.y + u % M;
    const int yp = min(y + 1, a.ny - 1), ym = max(y - 1, 0);
    const int xp = min(x + 1, a.nx - 1), xm = max(x - 1, 0);
    const float2 gy = cscale(csub(__ldg(a.O + (size_t)yp * a.nx + x), __ldg(a.O + (size_t)ym * a.nx + x)), 0.5f);
    const float2 gx = cscale(csub(__ldg(a.O + (size_t)y * a.nx + xp), __ldg(a.O + (size_t)y * a.nx + xm)), 0.5f);
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float2 pk = __ldg(Pj + (size_t)k * MM + u);
      const float2 xk = __ldcs(a.X + ((size_t)j * K + k) * MM + u);
      const float2 ay = cmul(pk, gy), ax = cmul(pk, gx);
      s0 += cabs2(ay);
      s1 += fmaf(ay.x, ax.x, ay.y * ax.y);
      s2 += cabs2(ax);
      s3 += fmaf(ay.x, xk.x, ay.y * xk.y);
      s4 += fmaf(ax.x, xk.x, ax.y * xk.y);
    }
  }
  const double A11 = block_sum_d<STEP_NT>(s0, red);
  const double A12 = block_sum_d<STEP_NT>(s1, red);
  const double A22 = block_sum_d<STEP_NT>(s2, red);
  const double r1 = block_sum_d<STEP_NT>(s3, red);
  const double r2 = block_sum_d<STEP_NT>(s4, red);
  if (threadIdx.x == 0) {
    double sy = 0.0, sx = 0.0;
    const double tr = A11 + A22;
    if (tr > 0.0) {
      const double lam = 1e-6 * tr / 2.0;
      const double a11 = A11 + lam, a22 = A22 + lam;
      const double det = a11 * a22 - A12 * A12;
      sy = (a22 * r1 - A12 * r2) / det;
      sx = (a11 * r2 - A12 * r1) / det;
    }
    a.out[j] = make_float2((float)sy, (float)sx);
  }
}

// Final fixed-order FP64 reduction of n (num, den) partials.
__global__ void __launch_bounds__(1024) k_err_final(const double2* part, int n, double2* out) {
  __shared__ double red[32];
  double sn = 0.0, sd = 0.0;
  for (int i = threadIdx.x; i < n; i += 1024) {
    sn += part[i].x;
    sd += part[i].y;
  }
  const double tn = block_sum_d<1024>(sn, red);
  const double td = block_sum_d<1024>(sd, red);
  if (threadIdx.x == 0) out[0] = make_double2(tn, td);
}

}  // namespace ptycho

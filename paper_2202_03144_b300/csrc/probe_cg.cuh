// Sub-pixel DM probe update: preconditioned conjugate gradients on
//     (B + d) P = sum_b T_-delta(b)[num_b] + d P_old,
//     B X = sum_b T_-delta(b)[Dbar_b T_delta(b) X],
// with Dbar_b = sum_{j in bin b} |O_j|^2 (per-bin sums of the probe pass),
// preconditioner W = den_P + d (den_P = sum_b Dbar_b), d = reg max den_P and
// the real inner product Re<x, y> over all modes and pixels.  B X is a
// shifted-table build of X scaled per bin (fused into the build) and an
// adjoint shift-sum (shift.cuh); the vector steps below fuse everything else.
//
// Every inner product is written as per-block FP64 partials; the next kernel
// adds them in block order in every block (deterministic, no atomics), so the
// whole solve is a fixed launch sequence with no host round trip.
#pragma once
#include "common.cuh"

namespace ptycho {

constexpr int CG_NT = 256;

struct CgArgs {
  float2* X;               // the probe, updated in place [K][MM]
  float2* r;               // residual
  float2* p;               // search direction
  const float2* q;         // B p (or B X at the start), from the shift-sum
  const float2* num;       // sum_b T_-delta(b)[num_b]
  const float* den;        // den_P [MM]
  const float* blk_max;    // block maxima of den_P [nblk_den]
  int nblk_den;
  float reg;
  int K, MM;
  double* part_rz;         // [2][nb] ping-pong partials of <r, z>
  double* part_pq;         // [nb] partials of <p, (B + d) p>
  int nb;                  // blocks of the vector kernels
  int it;                  // CG iteration (selects the ping-pong half)
};

__device__ __forceinline__ float cg_delta(const CgArgs& a, float* red, float* s) {
  float m = 0.f;
  for (int i = threadIdx.x; i < a.nblk_den; i += CG_NT) m = fmaxf(m, a.blk_max[i]);
  m = block_max_f<CG_NT>(m, red);
  if (threadIdx.x == 0) *s = a.reg * m;
  __syncthreads();
  return *s;
}

// Fixed-order sum of n partials, broadcast to the block.
__device__ __forceinline__ double cg_total(const double* part, int n, double* red, double* s) {
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += CG_NT) v += part[i];
  v = block_sum_d<CG_NT>(v, red);
  if (threadIdx.x == 0) *s = v;
  __syncthreads();
  const double t = *s;
  __syncthreads();
  return t;
}

__device__ __forceinline__ void cg_write_partial(double v, double* out, double* red) {
  v = block_sum_d<CG_NT>(v, red);
  if (threadIdx.x == 0) out[blockIdx.x] = v;
}

// r = num - B X (X = P_old, the proximal terms cancel), p = z = r / W.
__global__ void __launch_bounds__(CG_NT) k_cg_start(CgArgs a) {
  __shared__ float redf[32];
  __shared__ double redd[32];
  __shared__ float sd;
  const float d = cg_delta(a, redf, &sd);
  const int i = blockIdx.x * CG_NT + threadIdx.x;
  double rz = 0.0;
  if (i < a.K * a.MM) {
    const float2 r = csub(a.num[i], a.q[i]);
    const float w = a.den[i % a.MM] + d;
    const float2 z = w > 0.f ? cscale(r, 1.f / w) : make_float2(0.f, 0.f);
    a.r[i] = r;
    a.p[i] = z;
    rz = (double)r.x * z.x + (double)r.y * z.y;
  }
  cg_write_partial(rz, a.part_rz, redd);
}

// partials of <p, (B + d) p>
__global__ void __launch_bounds__(CG_NT) k_cg_pq(CgArgs a) {
  __shared__ float redf[32];
  __shared__ double redd[32];
  __shared__ float sd;
  const float d = cg_delta(a, redf, &sd);
  const int i = blockIdx.x * CG_NT + threadIdx.x;
  double pq = 0.0;
  if (i < a.K * a.MM) {
    const float2 p = a.p[i], q = a.q[i];
    pq = (double)p.x * (q.x + d * p.x) + (double)p.y * (q.y + d * p.y);
  }
  cg_write_partial(pq, a.part_pq, redd);
}

// alpha = <r,z> / <p,(B+d)p>;  X += alpha p;  r -= alpha (B+d) p;  partials of the new <r,z>
__global__ void __launch_bounds__(CG_NT) k_cg_step(CgArgs a) {
  __shared__ float redf[32];
  __shared__ double redd[32];
  __shared__ float sd;
  __shared__ double s;
  const float d = cg_delta(a, redf, &sd);
  const double* rz_old = a.part_rz + (size_t)(a.it & 1) * a.nb;
  double* rz_new = a.part_rz + (size_t)((a.it + 1) & 1) * a.nb;
  const double rz = cg_total(rz_old, a.nb, redd, &s);
  const double pq = cg_total(a.part_pq, a.nb, redd, &s);
  const float alpha = pq > 0.0 ? (float)(rz / pq) : 0.f;
  const int i = blockIdx.x * CG_NT + threadIdx.x;
  double v = 0.0;
  if (i < a.K * a.MM) {
    const float2 p = a.p[i], q = a.q[i];
    const float2 x = a.X[i];
    a.X[i] = make_float2(fmaf(alpha, p.x, x.x), fmaf(alpha, p.y, x.y));
    float2 r = a.r[i];
    r.x = fmaf(-alpha, fmaf(d, p.x, q.x), r.x);
    r.y = fmaf(-alpha, fmaf(d, p.y, q.y), r.y);
    a.r[i] = r;
    const float w = a.den[i % a.MM] + d;
    const float2 z = w > 0.f ? cscale(r, 1.f / w) : make_float2(0.f, 0.f);
    v = (double)r.x * z.x + (double)r.y * z.y;
  }
  cg_write_partial(v, rz_new, redd);
}

// beta = <r,z>_new / <r,z>_old;  p = z + beta p
__global__ void __launch_bounds__(CG_NT) k_cg_dir(CgArgs a) {
  __shared__ float redf[32];
  __shared__ double redd[32];
  __shared__ float sd;
  __shared__ double s;
  const float d = cg_delta(a, redf, &sd);
  const double rz_old = cg_total(a.part_rz + (size_t)(a.it & 1) * a.nb, a.nb, redd, &s);
  const double rz_new = cg_total(a.part_rz + (size_t)((a.it + 1) & 1) * a.nb, a.nb, redd, &s);
  const float beta = rz_old > 0.0 ? (float)(rz_new / rz_old) : 0.f;
  const int i = blockIdx.x * CG_NT + threadIdx.x;
  if (i < a.K * a.MM) {
    const float w = a.den[i % a.MM] + d;
    const float2 r = a.r[i];
    const float2 z = w > 0.f ? cscale(r, 1.f / w) : make_float2(0.f, 0.f);
    const float2 p = a.p[i];
    a.p[i] = make_float2(fmaf(beta, p.x, z.x), fmaf(beta, p.y, z.y));
  }
}

}  // namespace ptycho

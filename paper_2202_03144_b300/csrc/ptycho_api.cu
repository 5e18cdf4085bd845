// C ABI of the B300 ptychography engine (declared in include/ptycho.h).
//
// Host side of the library: parameter validation, device buffers, the CSR
// lists of positions per object tile, the ePIE visiting order, the kernel
// dispatch table and the per-iteration launch sequences of ePIE, DM and
// LSQML.  Every step of an iteration runs in the CUDA kernels of fourier.cuh,
// overlap.cuh and epie.cuh; nothing here computes on the host beyond the
// geometry (rounding positions, tile lists) and the random visiting order.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/ptycho.h"
#include "epie.cuh"
#include "fourier.cuh"
#include "fourier2.cuh"
#include "kernel_sets.cuh"
#include "modes.cuh"
#include "net.cuh"
#include "net_bwd_tc.cuh"
#include "overlap.cuh"
#include "shift.cuh"
#include "probe_cg.cuh"
#include "epie_sub.cuh"
#include "dft_tc.cuh"

namespace ptycho {
using TcFourierFn = void (*)(Fourier2Args, const unsigned char*, int);
TcFourierFn tc64_fourier(int mode, int istore);
void tc64_build_matrix(unsigned char* out, cudaStream_t st);
}  // namespace ptycho

using namespace ptycho;

// ---------------------------------------------------------------------------
// Kernel dispatch table: one entry per compiled (M, K, C).
// ---------------------------------------------------------------------------
namespace {

// The Fourier kernel variants of a set with their dynamic shared memory.
std::vector<std::pair<FourierFn, size_t>> fourier_variants(const KernelSet* ks) {
  std::vector<std::pair<FourierFn, size_t>> v{{ks->fourier, ks->smem_fourier}};
  for (int r = 0; r < 5; ++r)
    for (FourierFn f : ks->spec[r])
      if (f) v.push_back({f, ks->smem_row[r]});
  return v;
}

// Dynamic shared memory (and, above 8 CTAs, the non-portable cluster size)
// for every Fourier kernel variant of a set.
cudaError_t set_fourier_attributes(const KernelSet* ks) {
  cudaError_t e = cudaSuccess;
  for (auto [f, smem] : fourier_variants(ks)) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && ks->C > 8) e = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  }
  return e;
}

const std::vector<KernelSet>& kernel_sets() {
  static const std::vector<KernelSet> sets = [] {
    std::vector<KernelSet> v;
    for (auto part : {kernel_sets_16_32, kernel_sets_64, kernel_sets_128, kernel_sets_256, kernel_sets_mixed})
      for (const KernelSet& k : part()) v.push_back(k);
    return v;
  }();
  return sets;
}

const KernelSet* find_set(int M, int K, int C) {
  for (const auto& s : kernel_sets())
    if (s.M == M && s.K == K && s.C == C) return &s;
  return nullptr;
}

// Default cluster size: the smallest compiled C that keeps one CTA's share of
// a position at <= 32 KB of complex data (four CTAs per SM), else <= 64 KB,
// else the smallest compiled C.  (Measured at M = 256, K = 1: 16 CTAs per
// position beat 8 by 3%.)
int default_cluster(int M, int K) {
  auto ok = [&](int C) {
    const KernelSet* s = find_set(M, K, C);
    return s && s->default_ok;
  };
  for (long long cap : {4096LL, 8192LL})
    for (int C = 1; C <= 16; C *= 2)
      if ((long long)K * M * M / C <= cap && ok(C)) return C;
  for (int C = 1; C <= 16; C *= 2)
    if (ok(C)) return C;
  return 0;
}

// Kernel set of the ePIE sweep: the context's own when the caller chose the
// cluster size, else the compiled (M, K) set with the most CTAs whose ePIE
// kernel fits in shared memory (the sweep is latency-bound: more SMs per
// position, less time per position).
const KernelSet* epie_set(const ptycho_params* p, const KernelSet* own, int optin) {
  if (p->cluster > 0) return own;
  const KernelSet* best = nullptr;
  for (const auto& s : kernel_sets()) {
    const bool fits = (s.epie2 && s.smem_epie2 <= (size_t)optin) || (s.epie && s.smem_epie <= (size_t)optin);
    if (s.M == p->M && s.K == p->K && fits && (!best || s.C > best->C)) best = &s;
  }
  return best ? best : own;
}

thread_local std::string g_create_error;

__global__ void k_twiddle(float2* tw, int M) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) {
    double s, c;
    sincospi(2.0 * (double)i / (double)M, &s, &c);
    tw[i] = make_float2((float)c, (float)-s);
  }
}

// tw2[k1 * R2 + n2] = exp(-2 pi i n2 k1 / M), the inter-stage twiddles of
// the two-stage (R1 x R2) transforms of k_fourier2.
__global__ void k_twiddle2(float2* tw, int M, int R2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) {
    const int k1 = i / R2, n2 = i % R2;
    double s, c;
    sincospi(2.0 * (double)(n2 * k1) / (double)M, &s, &c);
    tw[i] = make_float2((float)c, (float)-s);
  }
}

// Detector-centred frames -> FFT order (the half-size roll of ifftshift) and
// sqrt(I), masked pixels (I < 0) -> -1, non-finite -> flag.  One block per
// (row, frame); V = 4 pixels per thread from 16-byte aligned sources (M is a
// multiple of 8, so a group of four never wraps around the roll), else 1.
template <int V>
__global__ void k_amp_f32(const float* __restrict__ src, int nj, int M, float* __restrict__ dst, int* bad) {
  const int ky = blockIdx.x, h = M / 2;
  const int sy = ky + h < M ? ky + h : ky + h - M;
  int b = 0;
  for (int j = blockIdx.y; j < nj; j += gridDim.y) {
    const float* srow = src + ((size_t)j * M + sy) * M;
    float* drow = dst + ((size_t)j * M + ky) * M;
    for (int kx = V * threadIdx.x; kx < M; kx += V * blockDim.x) {
      const int sx = kx + h < M ? kx + h : kx + h - M;
      float v[V];
      if constexpr (V == 4) {
        const float4 q = *reinterpret_cast<const float4*>(srow + sx);
        v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
      } else {
        v[0] = srow[sx];
      }
#pragma unroll
      for (int e = 0; e < V; ++e) {
        b |= !isfinite(v[e]);
        v[e] = v[e] < 0.f ? -1.f : sqrtf(v[e]);
      }
      if constexpr (V == 4) *reinterpret_cast<float4*>(drow + kx) = make_float4(v[0], v[1], v[2], v[3]);
      else drow[kx] = v[0];
    }
  }
  if (b) *bad = 1;
}

// Per-frame maximum of sqrt(I) (masked pixels ignored); one CTA per frame.
__global__ void __launch_bounds__(256) k_frame_max(const float* __restrict__ src, int M, float* out, int* bad) {
  __shared__ float red[32];
  const size_t MM = (size_t)M * M;
  const float* f = src + blockIdx.x * MM;
  float m = 0.f;
  for (size_t i = threadIdx.x; i < MM; i += 256) {
    const float v = f[i];
    if (!isfinite(v)) *bad = 1;
    if (v > 0.f) m = fmaxf(m, sqrtf(v));
  }
  m = block_max_f<256>(m, red);
  if (threadIdx.x == 0) out[blockIdx.x] = m > 0.f ? m : 1.f;
}

template <typename T>
__device__ __forceinline__ T to16(float v);
template <>
__device__ __forceinline__ __half to16<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 to16<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// 16-bit storage: sqrt(I) / s_j rounded to the format; same layout as k_amp_f32.
template <typename T, int V>
__global__ void k_amp_q16(const float* __restrict__ src, int nj, int M, const float* __restrict__ scale,
                          T* __restrict__ dst) {
  const int ky = blockIdx.x, h = M / 2;
  const int sy = ky + h < M ? ky + h : ky + h - M;
  for (int j = blockIdx.y; j < nj; j += gridDim.y) {
    const float* srow = src + ((size_t)j * M + sy) * M;
    T* drow = dst + ((size_t)j * M + ky) * M;
    const float sc = scale[j];
    for (int kx = V * threadIdx.x; kx < M; kx += V * blockDim.x) {
      const int sx = kx + h < M ? kx + h : kx + h - M;
      float v[V];
      if constexpr (V == 4) {
        const float4 q = *reinterpret_cast<const float4*>(srow + sx);
        v[0] = q.x, v[1] = q.y, v[2] = q.z, v[3] = q.w;
      } else {
        v[0] = srow[sx];
      }
#pragma unroll
      for (int e = 0; e < V; ++e) drow[kx + e] = to16<T>(v[e] < 0.f ? -1.f : sqrtf(v[e]) / sc);
    }
  }
}

// Detector preprocessing of nj raw frames [H][W] into detector-centred
// M x M intensities: output offset d = (y - M/2, x - M/2) reads raw pixel
// (cy, cx) + R^-rot d (R: quarter turn counter-clockwise, (a, b) -> (-b, a)),
// offsets wrapped into [-M/2, M/2); outside the frame, negative or >= sat:
// masked (-1); below thr (> 0): 0; NaN/Inf raise *bad.  One block per
// (output row, frame).
struct PreArgs {
  const void* raw;
  int nj, H, W, cy, cx, M, rot;
  float sat, thr;
  float* out;
  int* bad;
};

template <typename T>
__global__ void k_preprocess(PreArgs a) {
  const int y = blockIdx.x, h = a.M / 2;
  const T* raw = reinterpret_cast<const T*>(a.raw);
  int b = 0;
  for (int f = blockIdx.y; f < a.nj; f += gridDim.y) {
    for (int x = threadIdx.x; x < a.M; x += blockDim.x) {
      int sy = y - h, sx = x - h;
      for (int k = 0; k < a.rot; ++k) {  // R^-1: (a, b) -> (b, -a)
        const int t = sy;
        sy = sx;
        sx = -t;
      }
      sy = ((sy + h) % a.M + a.M) % a.M - h;
      sx = ((sx + h) % a.M + a.M) % a.M - h;
      const int ry = a.cy + sy, rx = a.cx + sx;
      float v = -1.f;
      if (ry >= 0 && ry < a.H && rx >= 0 && rx < a.W) {
        v = (float)raw[((size_t)f * a.H + ry) * a.W + rx];
        b |= !isfinite(v);
        if (v < 0.f || v >= a.sat) v = -1.f;
        else if (a.thr > 0.f && v < a.thr) v = 0.f;
      }
      a.out[((size_t)f * a.M + y) * a.M + x] = v;
    }
  }
  if (b) *a.bad = 1;
}

// Raise *bad if any of n floats is NaN or Inf.
__global__ void k_check_finite(const float* __restrict__ p, size_t n, int* bad) {
  int b = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    b |= !isfinite(p[i]);
  if (__syncthreads_or(b) && threadIdx.x == 0) *bad = 1;
}

__global__ void k_fill_c(float2* p, size_t n, float2 v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

// psi_{j,k} = P_k O_j (DM initial state)
__global__ void k_exit_waves(const float2* __restrict__ O, int nx, const float2* __restrict__ P,
                             const unsigned short* __restrict__ pbin, const int2* __restrict__ pos, int J, int K,
                             int M, float2* __restrict__ X) {
  const size_t MM = (size_t)M * M;
  const size_t n = (size_t)J * K * MM;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t u = i % MM;
    const int k = (int)((i / MM) % K);
    const int j = (int)(i / (MM * K));
    const int2 p = pos[j];
    const int uy = (int)(u / M), ux = (int)(u % M);
    const size_t b = pbin ? pbin[j] : 0;
    X[i] = cmul(P[(b * K + k) * MM + u], O[(size_t)(p.x + uy) * nx + p.y + ux]);
  }
}

// SplitMix64 (Steele, Lea & Flood) -- the counter-based generator that
// drives the ePIE visiting order.
struct SplitMix64 {
  uint64_t s;
  uint64_t next() {
    s += 0x9E3779B97F4A7C15ull;
    uint64_t z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
};

}  // namespace

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct ptycho_ctx {
  ptycho_params p{};
  cudaStream_t st = nullptr;
  const KernelSet* ks = nullptr;
  const KernelSet* eks = nullptr;  // kernel set of the ePIE sweep
  const KernelSet* fks_one = nullptr;  // Fourier kernels of one-position passes (sub-pixel ePIE)
  const KernelSet* f_ks = nullptr;     // set by a pass that overrides ks
  int C = 1;
  // device state
  float2* O = nullptr;
  float2* P = nullptr;
  float2* X = nullptr;       // DM exit waves psi / LSQML residual chi [J][K][M][M]
  float2* dO = nullptr;      // LSQML object direction
  float2* dP = nullptr;      // LSQML probe direction
  float2* tw = nullptr;
  float2* tw2 = nullptr;
  int* err_flag = nullptr;   // set by a device wait that gave up
  int wait_limit = 1 << 20;  // polls of a cluster-transpose wait (ptycho_set_wait_limit)
  bool x16 = false;          // inside an LSQML iteration with FP16 residual storage
  cudaStream_t st_side = nullptr;  // second stream: the probe-direction sums beside the object's
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  unsigned char* dftm = nullptr;  // split DFT matrix of the tensor-core engine
  int n_sm = 0;
  size_t mem_used = 0;       // device bytes allocated by dalloc and not yet freed
  std::unordered_map<void*, size_t> mem_blocks;
  int2* pos = nullptr;
  void* amp = nullptr;       // stored sqrt(I)
  float* amp_scale = nullptr;
  float* denO = nullptr;
  float* tile_max = nullptr;
  float* denO_max = nullptr;
  int* tile_ptr = nullptr;
  int* tile_list = nullptr;
  size_t tile_list_cap = 0;   // ints allocated for tile_list
  int n_tiles = 0, ntx = 0, nty = 0;
  int G = 1;                 // position groups of the probe sums
  int G_cap = 1;             // capacity of the group partials
  // sub-pixel positions (S = params.subpixel > 0): per-position bin of the
  // shifted-probe table, the tables of P and dP, per-bin probe sums, the
  // line-shift scratch, and the probe-sum groups in bin order
  int S = 0;
  int G_sub = 0;             // groups in bin order (sub-pixel)
  unsigned short* pbin = nullptr;
  float2* Pt = nullptr;
  float2* dPt = nullptr;
  float2* pbins = nullptr;
  float2* stmp = nullptr;
  int* porder = nullptr;
  int* goff = nullptr;
  int* bgrp = nullptr;
  float* pbins_den = nullptr;  // per-bin den_P (the DM probe solve)
  float2* cg_r = nullptr;      // DM probe solve: residual, direction, operator output
  float2* cg_p = nullptr;
  float2* cg_q = nullptr;
  double* cg_part = nullptr;   // [3][blocks] inner-product partials
  float2* pos_corr = nullptr;  // position refinement: per-position shift
  float2* ep_mx = nullptr;     // sub-pixel ePIE: partial maxima
  // position blocks (params.block_positions = B > 0, LSQML): X holds the
  // residuals of B positions; blk is the block the launches work on
  int B = 0;
  float2* objacc = nullptr;    // accumulated alpha-weighted object numerator
  struct Block {
    bool on = false;
    int j0 = 0, n = 0;
    bool accumulate = false;
  } blk;
  // a Fourier pass with an explicit probe (no table) and residual offset:
  // the sub-pixel ePIE sweep, one position at a time
  const float2* f_P = nullptr;
  int f_xoff = -1;
  std::vector<unsigned short> bin_host;  // sub-pixel bin of each position
  std::vector<float> pos_f;    // positions as last set (or refined), [J][2]
  float2* ppart = nullptr;
  float* ppart_den = nullptr;
  float2* pnum = nullptr;
  float* pden = nullptr;
  float* pblk_max = nullptr;
  float* alphaO = nullptr;
  float* alphaP = nullptr;
  double2* gram = nullptr;   // probe-mode Gram matrix [K][K]
  double2* modeV = nullptr;  // its eigenvectors [K][K] (orthogonalisation)
  double2* err_part = nullptr;
  double2* err_out = nullptr;
  int* order = nullptr;
  int order_cap = 0;
  int* flag = nullptr;
  // upload staging (host inputs): two halves of stage_bytes / 2, filled on
  // st_copy while the kernels of the other half run on st
  float* stage = nullptr;
  size_t stage_bytes = 0;
  float* pre = nullptr;      // preprocessed detector-centred frames of one chunk
  int pre_frames = 0;
  cudaStream_t st_copy = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr}, ev_used[2] = {nullptr, nullptr};
  // host-side state
  bool have_pos = false, have_data = false;
  bool epie_ok = false;    // the ePIE kernel of this (M, K, C) fits in shared memory
  bool epie2 = false;      // ... and it is the register-resident form (k_epie2)
  bool psi_valid = false;  // X holds the DM state
  long long t = 0;
  long long launches = 0;
  std::string err;
  // logging (ptycho_set_log)
  ptycho_log_fn log_fn = nullptr;
  void* log_user = nullptr;
  int log_every = 0;
  // profiling
  struct Pending {
    int fam;
    cudaEvent_t a, b;
    double bytes;
  };
  bool prof = false;
  bool pdl = false;   // launch with programmatic stream serialization (chains of small kernels)
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::string> fam_names;
  std::vector<ptycho_kernel_stat> stats;
  std::vector<int2> pos_host;
};

namespace {

int fail(ptycho_ctx* c, int code, const char* fmt, ...) {
  char b[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(b, sizeof b, fmt, ap);
  va_end(ap);
  if (c) {
    c->err = b;
    if (c->log_fn) c->log_fn(c->log_user, PTYCHO_LOG_ERROR, b);
  } else {
    g_create_error = b;
  }
  return code;
}

// NVTX range (host timeline of a profiler; no-op without one attached)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? PTYCHO_ERR_OOM : PTYCHO_ERR_CUDA,    \
                  "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);       \
  } while (0)

template <typename T>
int dalloc(ptycho_ctx* ctx, T** p, size_t n) {
  if (*p) return 0;
  const size_t bytes = n * sizeof(T) + 16;
  if (ctx->p.mem_limit && ctx->mem_used + bytes > ctx->p.mem_limit)
    return fail(ctx, PTYCHO_ERR_OOM, "allocation of %zu bytes would pass the context's device memory limit (%zu of %llu bytes in use)",
                bytes, ctx->mem_used, ctx->p.mem_limit);
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    cudaGetLastError();
    return fail(ctx, PTYCHO_ERR_OOM, "cudaMalloc of %zu bytes failed: %s", n * sizeof(T), cudaGetErrorString(e));
  }
  ctx->mem_used += bytes;
  ctx->mem_blocks[(void*)*p] = bytes;
  return 0;
}

// Free a buffer from dalloc (NULL is ignored) and return its bytes to the
// context's budget.
template <typename T>
void dfree(ptycho_ctx* ctx, T*& p) {
  if (!p) return;
  auto it = ctx->mem_blocks.find((void*)p);
  if (it != ctx->mem_blocks.end()) {
    ctx->mem_used -= it->second;
    ctx->mem_blocks.erase(it);
  }
  cudaFree((void*)p);
  p = nullptr;
}

// Staging buffer of at least `bytes`, the copy stream and its events.
int ensure_stage(ptycho_ctx* ctx, size_t bytes) {
  if (ctx->stage_bytes < bytes) {
    if (ctx->stage) {
      CK(cudaStreamSynchronize(ctx->st));
      if (ctx->st_copy) CK(cudaStreamSynchronize(ctx->st_copy));
      dfree(ctx, ctx->stage);
      ctx->stage_bytes = 0;
    }
    if (int r = dalloc(ctx, &ctx->stage, bytes / 4 + 1)) return r;
    ctx->stage_bytes = bytes;
  }
  if (!ctx->st_copy) {
    CK(cudaStreamCreateWithFlags(&ctx->st_copy, cudaStreamNonBlocking));
    for (int h = 0; h < 2; ++h) {
      CK(cudaEventCreateWithFlags(&ctx->ev_copied[h], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&ctx->ev_used[h], cudaEventDisableTiming));
    }
  }
  return 0;
}

cudaEvent_t get_event(ptycho_ctx* ctx) {
  if (!ctx->ev_pool.empty()) {
    cudaEvent_t e = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

int family(ptycho_ctx* ctx, const char* name) {
  for (size_t i = 0; i < ctx->fam_names.size(); ++i)
    if (ctx->fam_names[i] == name) return (int)i;
  ctx->fam_names.push_back(name);
  ptycho_kernel_stat s{};
  ctx->stats.push_back(s);
  return (int)ctx->fam_names.size() - 1;
}

// Launch wrapper: counts launches, optionally brackets them with events and
// checks the launch error.
template <class Fn>
int launch(ptycho_ctx* ctx, const char* name, double bytes, Fn&& fn) {
  NvtxRange range(name);
  ptycho_ctx::Pending rec{};
  if (ctx->prof) {
    rec.fam = family(ctx, name);
    rec.a = get_event(ctx);
    rec.b = get_event(ctx);
    rec.bytes = bytes;
    cudaEventRecord(rec.a, ctx->st);
  }
  fn();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(ctx, PTYCHO_ERR_CUDA, "launch of %s failed: %s", name, cudaGetErrorString(e));
  ctx->launches++;
  if (ctx->prof) {
    cudaEventRecord(rec.b, ctx->st);
    ctx->pending.push_back(rec);
  }
  return 0;
}

// A kernel launch on the context's stream, with programmatic stream
// serialization when ctx->pdl is set (the kernel then calls pdl_wait() before
// touching what its predecessor writes or reads).
template <class... KArgs, class... Args>
void launch_k(ptycho_ctx* ctx, void (*kern)(KArgs...), dim3 grid, dim3 block, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.stream = ctx->st;
  cudaLaunchAttribute attr[1];
  if (ctx->pdl) {
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  cudaLaunchKernelEx(&cfg, kern, args...);
}

int collect_profile(ptycho_ctx* ctx) {
  if (ctx->pending.empty()) return 0;
  CK(cudaStreamSynchronize(ctx->st));
  for (auto& r : ctx->pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    auto& s = ctx->stats[r.fam];
    s.launches++;
    s.ms += ms;
    s.bytes += r.bytes;
    ctx->ev_pool.push_back(r.a);
    ctx->ev_pool.push_back(r.b);
  }
  ctx->pending.clear();
  return 0;
}

size_t amp_bytes(const ptycho_ctx* ctx) { return ctx->p.istore == PTYCHO_I_F32 ? 4 : 2; }

// ----------------------------------------------------------------- Fourier
int launch_shift(ptycho_ctx* ctx, bool build, const float2* src, float2* dst, const float* bscale = nullptr);
int refresh_probe_table(ptycho_ctx* ctx);
const float2* probe_view(const ptycho_ctx* ctx);
const unsigned short* bin_view(const ptycho_ctx* ctx);

// Every Fourier pass reads the probe as it is now: with sub-pixel positions
// the shifted table is rebuilt first.
int launch_fourier(ptycho_ctx* ctx, int mode, float2* X, float* I_out, int j0, int nj, const char* name) {
  if (!ctx->f_P)
    if (int r = refresh_probe_table(ctx)) return r;
  const KernelSet* ks = ctx->f_ks ? ctx->f_ks : ctx->ks;
  Fourier2Args a{};
  a.O = ctx->O;
  a.nx = ctx->p.obj_nx;
  a.P = ctx->f_P ? ctx->f_P : probe_view(ctx);
  a.pbin = ctx->f_P ? nullptr : bin_view(ctx);
  a.pos = ctx->pos;
  a.X = X;
  a.amp = ctx->amp;
  a.amp_scale = ctx->amp_scale;
  a.istore = ctx->p.istore;
  a.I_out = I_out;
  a.err_part = ctx->err_part;
  a.tw2 = ctx->tw2;
  a.err_flag = ctx->err_flag;
  a.wait_limit = ctx->wait_limit;
  a.x16 = ctx->x16 && X == ctx->X && (mode == FM_CHI || mode == FM_CHIP);
  a.j0 = j0;
  a.nj = nj;
  a.xoff = ctx->f_xoff >= 0 ? ctx->f_xoff : ((ctx->blk.on && X == ctx->X) ? ctx->blk.j0 : 0);
  a.mode = mode;
  const double MM = (double)ctx->p.M * ctx->p.M;
  const double K = ctx->p.K;
  double bytes = 0;
  switch (mode) {
    case FM_DM: bytes = nj * MM * (16.0 * K + amp_bytes(ctx)); break;
    case FM_CHI:
    case FM_CHIP: bytes = nj * MM * ((a.x16 ? 4.0 : 8.0) * K + amp_bytes(ctx)); break;
    case FM_ERR: bytes = nj * MM * amp_bytes(ctx); break;
    case FM_SIM: bytes = nj * MM * 4.0; break;
  }
  if (ctx->p.fft_engine == PTYCHO_DFT_TENSOR_BF16X3) {
    // tensor-core DFT: persistent CTAs, two per SM
    const TcFourierFn fn = tc64_fourier(mode, a.istore);
    if (!fn) return fail(ctx, PTYCHO_ERR_UNSUPPORTED, "no tensor-core Fourier kernel for mode %d", mode);
    const int grid = std::max(1, std::min(nj, 2 * ctx->n_sm));
    return launch(ctx, name, bytes, [&] {
      fn<<<grid, TC64_NT, TC64_SMEM, ctx->st>>>(a, ctx->dftm, ctx->C);
    });
  }
  return launch(ctx, name, bytes, [&] {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)(ks->C * nj));
    cfg.blockDim = dim3((unsigned)ks->NT2);
    cfg.dynamicSmemBytes = ks->smem_fourier;
    cfg.stream = ctx->st;
    cudaLaunchAttribute attr[2];
    unsigned na = 0;
    if (ks->C > 1) {
      attr[na].id = cudaLaunchAttributeClusterDimension;
      attr[na].val.clusterDim.x = ks->C;
      attr[na].val.clusterDim.y = 1;
      attr[na].val.clusterDim.z = 1;
      ++na;
    }
    if (ctx->pdl) {
      attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
      attr[na].val.programmaticStreamSerializationAllowed = 1;
      ++na;
    }
    cfg.attrs = na ? attr : nullptr;
    cfg.numAttrs = na;
    FourierFn fn = ks->fourier;
    const int row = spec_row(mode);
    if (row >= 0 && a.istore >= 0 && a.istore < 3 && ks->spec[row][a.istore]) {
      fn = ks->spec[row][a.istore];
      cfg.dynamicSmemBytes = ks->smem_row[row];
    }
    cudaLaunchKernelEx(&cfg, fn, a);
  });
}

int check_device_flag(ptycho_ctx* ctx) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, ctx->err_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (h) {
    cudaMemsetAsync(ctx->err_flag, 0, sizeof(int), ctx->st);
    return fail(ctx, PTYCHO_ERR_TIMEOUT, "a bounded device wait gave up (bulk copy did not complete)");
  }
  return 0;
}

// ------------------------------------------------------ sub-pixel shifts
template <int M>
int launch_shift_m(ptycho_ctx* ctx, bool build, const float2* src, float2* dst, const float* bscale) {
  constexpr int LN = 8;
  const int K = ctx->p.K, S = ctx->S;
  const double tab = 8.0 * S * S * K * (double)M * M;
  if (build) {
    if (int r = launch(ctx, "shift_build", tab, [&] {
          k_shift_build_rows<M, LN><<<dim3(K * M / LN, S), SH_NT, 0, ctx->st>>>(src, ctx->stmp, K, S, ctx->tw, 0, 0);
          k_shift_build_cols<M, LN><<<dim3(M / LN, K, S * S), SH_NT, 0, ctx->st>>>(ctx->stmp, dst, K, S, ctx->tw, 0,
                                                                                 0, 0, bscale);
        }))
      return r;
    return 0;
  }
  return launch(ctx, "shift_sum", tab, [&] {
    k_shift_sum_cols<M, LN><<<dim3(M / LN, K, S), SH_NT, 0, ctx->st>>>(src, ctx->stmp, K, S, ctx->bgrp, ctx->tw);
    k_shift_sum_rows<M, LN><<<dim3(K * M / LN), SH_NT, 0, ctx->st>>>(ctx->stmp, dst, K, S, ctx->tw);
  });
}

// One shift: dst[k] = T_delta src[k], delta = (bye - S/2, bxe - S/2) / S
// (src and dst may be the same array: the row pass goes through stmp).
template <int M>
int launch_shift_one_m(ptycho_ctx* ctx, int bye, int bxe, const float2* src, float2* dst) {
  // one probe's shift is latency-bound: the fewest lines per CTA that still
  // give every thread an element (LN M a multiple of the block size)
  constexpr int LN = SH_NT / std::gcd(M, SH_NT);
  const int K = ctx->p.K, S = ctx->S;
  return launch(ctx, "shift_one", 16.0 * K * (double)M * M, [&] {
    launch_k(ctx, k_shift_build_rows<M, LN>, dim3(K * M / LN, 1), dim3(SH_NT), src, (float2*)ctx->stmp, K, S,
             (const float2*)ctx->tw, 1, bxe);
    launch_k(ctx, k_shift_build_cols<M, LN>, dim3(M / LN, K, 1), dim3(SH_NT), (const float2*)ctx->stmp, dst, K, S,
             (const float2*)ctx->tw, 1, bye, 0, (const float*)nullptr);
  });
}

int launch_shift_one(ptycho_ctx* ctx, int bye, int bxe, const float2* src, float2* dst) {
  switch (ctx->p.M) {
    case 16: return launch_shift_one_m<16>(ctx, bye, bxe, src, dst);
    case 32: return launch_shift_one_m<32>(ctx, bye, bxe, src, dst);
    case 64: return launch_shift_one_m<64>(ctx, bye, bxe, src, dst);
    case 96: return launch_shift_one_m<96>(ctx, bye, bxe, src, dst);
    case 128: return launch_shift_one_m<128>(ctx, bye, bxe, src, dst);
    case 192: return launch_shift_one_m<192>(ctx, bye, bxe, src, dst);
    case 256: return launch_shift_one_m<256>(ctx, bye, bxe, src, dst);
    default: return fail(ctx, PTYCHO_ERR_UNSUPPORTED, "sub-pixel shifts are not compiled for M=%d", ctx->p.M);
  }
}

// The frame change of the sub-pixel ePIE sweep: P = T_delta P in place,
// delta = (bye - S/2, bxe - S/2) / S, and the partial maxima of the step at
// position j (sum_k |P_k|^2 of the shifted probe, |O_j|^2) into mx; *nmx is
// their count.
template <int M, int K>
int launch_frame_change_m(ptycho_ctx* ctx, int bye, int bxe, int j, float2* mx, int* nmx) {
  constexpr int LN = SH_NT / std::gcd(M, SH_NT);
  static_assert(M / LN <= EPS_MX_CAP, "partial maxima buffer");
  const int S = ctx->S;
  *nmx = M / LN;
  return launch(ctx, "shift_one", 16.0 * K * (double)M * M, [&] {
    launch_k(ctx, k_shift_build_rows<M, LN>, dim3(K * M / LN, 1), dim3(SH_NT), (const float2*)ctx->P,
             (float2*)ctx->stmp, K, S, (const float2*)ctx->tw, 1, bxe);
    launch_k(ctx, k_shift_one_cols<M, LN, K>, dim3(M / LN), dim3(SH_NT), (const float2*)ctx->stmp, ctx->P, S,
             (const float2*)ctx->tw, bye, (const float2*)ctx->O, ctx->p.obj_nx, (const int2*)ctx->pos, j, mx);
  });
}

template <int K>
int launch_frame_change(ptycho_ctx* ctx, int bye, int bxe, int j, float2* mx, int* nmx) {
  switch (ctx->p.M) {
    case 16: return launch_frame_change_m<16, K>(ctx, bye, bxe, j, mx, nmx);
    case 32: return launch_frame_change_m<32, K>(ctx, bye, bxe, j, mx, nmx);
    case 64: return launch_frame_change_m<64, K>(ctx, bye, bxe, j, mx, nmx);
    case 96: return launch_frame_change_m<96, K>(ctx, bye, bxe, j, mx, nmx);
    case 128: return launch_frame_change_m<128, K>(ctx, bye, bxe, j, mx, nmx);
    case 192: return launch_frame_change_m<192, K>(ctx, bye, bxe, j, mx, nmx);
    case 256: return launch_frame_change_m<256, K>(ctx, bye, bxe, j, mx, nmx);
    default: return fail(ctx, PTYCHO_ERR_UNSUPPORTED, "sub-pixel shifts are not compiled for M=%d", ctx->p.M);
  }
}

// build: dst[bin][k] = T_delta(bin) src[k] (times bscale[bin] if given);
// sum: dst[k] = sum_bin T_-delta(bin) src[bin][k]
int launch_shift(ptycho_ctx* ctx, bool build, const float2* src, float2* dst, const float* bscale) {
  switch (ctx->p.M) {
    case 16: return launch_shift_m<16>(ctx, build, src, dst, bscale);
    case 32: return launch_shift_m<32>(ctx, build, src, dst, bscale);
    case 64: return launch_shift_m<64>(ctx, build, src, dst, bscale);
    case 96: return launch_shift_m<96>(ctx, build, src, dst, bscale);
    case 128: return launch_shift_m<128>(ctx, build, src, dst, bscale);
    case 192: return launch_shift_m<192>(ctx, build, src, dst, bscale);
    case 256: return launch_shift_m<256>(ctx, build, src, dst, bscale);
    default: return fail(ctx, PTYCHO_ERR_UNSUPPORTED, "sub-pixel shifts are not compiled for M=%d", ctx->p.M);
  }
}

// The shifted-probe table of the current probe (sub-pixel positions only).
int refresh_probe_table(ptycho_ctx* ctx) {
  return ctx->S ? launch_shift(ctx, true, ctx->P, ctx->Pt) : 0;
}
const float2* probe_view(const ptycho_ctx* ctx) { return ctx->S ? ctx->Pt : ctx->P; }
const unsigned short* bin_view(const ptycho_ctx* ctx) { return ctx->S ? ctx->pbin : nullptr; }

// ---------------------------------------------------------------- overlap
// object-side modes of obj_step (OBJ_UPD is the LSQML update)
constexpr int OBJ_STEP_DM = 100;   // DM overlap update of O
constexpr int OBJ_STEP_DIR = 101;  // LSQML direction dO
constexpr int OBJ_STEP_ACC = 102;  // position blocks: accumulate the weighted numerator in objacc

template <int K>
int launch_obj(ptycho_ctx* ctx, int mode, const float2* X, const float* w) {
  ObjArgs a{};
  a.O = ctx->O;
  a.dO = ctx->dO;
  a.ny = ctx->p.obj_ny;
  a.nx = ctx->p.obj_nx;
  a.ntx = ctx->ntx;
  a.P = probe_view(ctx);
  a.pbin = bin_view(ctx);
  a.X = X;
  a.pos = ctx->pos;
  a.tile_ptr = ctx->tile_ptr;
  a.tile_list = ctx->tile_list;
  a.weights = w;
  a.den = ctx->denO;
  a.tile_max = ctx->tile_max;
  a.den_max = ctx->denO_max;
  a.reg = (float)ctx->p.reg;
  a.beta = (float)ctx->p.lsqml_beta;
  a.M = ctx->p.M;
  const int nj = ctx->blk.on ? ctx->blk.n : ctx->p.J;
  if (ctx->blk.on) {
    a.jlo = ctx->blk.j0;
    a.jhi = ctx->blk.j0 + ctx->blk.n;
    a.xoff = ctx->blk.j0;
    a.accumulate = ctx->blk.accumulate;
  }
  const double obj = (double)ctx->p.obj_ny * ctx->p.obj_nx;
  const double xb = (ctx->x16 && X == ctx->X ? 4.0 : 8.0) * nj * K * (double)ctx->p.M * ctx->p.M;
  const dim3 g(ctx->n_tiles), b(OBJ_NT);
  const bool sub = ctx->S != 0;
  const bool h = ctx->x16 && X == ctx->X;  // FP16 residuals
  auto go = [&](auto kern) { kern<<<g, b, 0, ctx->st>>>(a); };
  if (mode == OBJ_STEP_ACC) {  // numerator only, into objacc
    a.dO = ctx->objacc;
    a.den = nullptr;
    return launch(ctx, "obj_update", xb + obj * 16.0, [&] {
      if (sub) go(h ? k_obj<K, OBJ_NUMDEN, true, __half2> : k_obj<K, OBJ_NUMDEN, true>);
      else go(h ? k_obj<K, OBJ_NUMDEN, false, __half2> : k_obj<K, OBJ_NUMDEN, false>);
    });
  }
  if (mode == OBJ_UPD)
    return launch(ctx, "obj_update", xb + obj * 20.0, [&] {
      if (sub) go(h ? k_obj<K, OBJ_UPD, true, __half2> : k_obj<K, OBJ_UPD, true>);
      else go(h ? k_obj<K, OBJ_UPD, false, __half2> : k_obj<K, OBJ_UPD, false>);
    });
  // numerator + den_O in one pass, then the max of den_O, then the epilogue
  if (int r = launch(ctx, "obj_sums", xb + obj * 12.0, [&] {
        if (sub) go(h ? k_obj<K, OBJ_NUMDEN, true, __half2> : k_obj<K, OBJ_NUMDEN, true>);
        else go(h ? k_obj<K, OBJ_NUMDEN, false, __half2> : k_obj<K, OBJ_NUMDEN, false>);
      }))
    return r;
  if (ctx->blk.on) return 0;  // the epilogue runs once, after the last block (obj_finish)
  if (int r = launch(ctx, "reduce_max", 0.0,
                     [&] { k_reduce_max<<<1, 1024, 0, ctx->st>>>(ctx->tile_max, ctx->n_tiles, ctx->denO_max); }))
    return r;
  const size_t n = (size_t)ctx->p.obj_ny * ctx->p.obj_nx;
  if (mode == OBJ_STEP_DM)
    return launch(ctx, "obj_norm", obj * 28.0, [&] {
      k_obj_norm<NORM_DM><<<1184, 256, 0, ctx->st>>>(ctx->O, ctx->dO, ctx->denO, ctx->denO_max, a.reg, n);
    });
  return launch(ctx, "obj_norm", obj * 20.0, [&] {
    k_obj_norm<NORM_DIR><<<1184, 256, 0, ctx->st>>>(ctx->O, ctx->dO, ctx->denO, ctx->denO_max, a.reg, n);
  });
}

// After the last position block: max of den_O and the direction (or the DM update).
int obj_finish(ptycho_ctx* ctx, int mode) {
  if (int r = launch(ctx, "reduce_max", 0.0,
                     [&] { k_reduce_max<<<1, 1024, 0, ctx->st>>>(ctx->tile_max, ctx->n_tiles, ctx->denO_max); }))
    return r;
  const size_t n = (size_t)ctx->p.obj_ny * ctx->p.obj_nx;
  const float reg = (float)ctx->p.reg;
  if (mode == OBJ_STEP_DM)
    return launch(ctx, "obj_norm", n * 28.0, [&] {
      k_obj_norm<NORM_DM><<<1184, 256, 0, ctx->st>>>(ctx->O, ctx->dO, ctx->denO, ctx->denO_max, reg, n);
    });
  return launch(ctx, "obj_norm", n * 20.0, [&] {
    k_obj_norm<NORM_DIR><<<1184, 256, 0, ctx->st>>>(ctx->O, ctx->dO, ctx->denO, ctx->denO_max, reg, n);
  });
}

int obj_step(ptycho_ctx* ctx, int mode, const float2* X, const float* w) {
  switch (ctx->p.K) {
    case 1: return launch_obj<1>(ctx, mode, X, w);
    case 2: return launch_obj<2>(ctx, mode, X, w);
    default: return launch_obj<3>(ctx, mode, X, w);
  }
}


// Sub-pixel DM probe update: DM_PROBE_CG iterations of preconditioned
// conjugate gradients on the probe's normal equations (probe_cg.cuh), from
// the current probe; pnum, pden, pbins_den and pblk_max come from the probe
// sums of this iteration.
constexpr int DM_PROBE_CG = 4;

// q = B v = sum_b T_-delta(b)[Dbar_b T_delta(b) v] (the scaling fused into the build)
int probe_normal_op(ptycho_ctx* ctx, const float2* v, float2* q) {
  if (int r = launch_shift(ctx, true, v, ctx->dPt, ctx->pbins_den)) return r;
  return launch_shift(ctx, false, ctx->dPt, q);
}

int dm_probe_cg(ptycho_ctx* ctx) {
  const int K = ctx->p.K, MM = ctx->p.M * ctx->p.M;
  CgArgs a{};
  a.X = ctx->P;
  a.r = ctx->cg_r;
  a.p = ctx->cg_p;
  a.q = ctx->cg_q;
  a.num = ctx->pnum;
  a.den = ctx->pden;
  a.blk_max = ctx->pblk_max;
  a.nblk_den = (MM + PROBE_NT - 1) / PROBE_NT;
  a.reg = (float)ctx->p.reg;
  a.K = K;
  a.MM = MM;
  a.nb = (K * MM + CG_NT - 1) / CG_NT;
  a.part_rz = ctx->cg_part;
  a.part_pq = ctx->cg_part + 2 * (size_t)a.nb;
  if (int r = probe_normal_op(ctx, ctx->P, ctx->cg_q)) return r;
  if (int r = launch(ctx, "probe_cg", 0.0, [&] { k_cg_start<<<a.nb, CG_NT, 0, ctx->st>>>(a); })) return r;
  for (int it = 0; it < DM_PROBE_CG; ++it) {
    a.it = it;
    if (int r = probe_normal_op(ctx, ctx->cg_p, ctx->cg_q)) return r;
    if (int r = launch(ctx, "probe_cg", 0.0, [&] {
          k_cg_pq<<<a.nb, CG_NT, 0, ctx->st>>>(a);
          k_cg_step<<<a.nb, CG_NT, 0, ctx->st>>>(a);
          k_cg_dir<<<a.nb, CG_NT, 0, ctx->st>>>(a);
        }))
      return r;
  }
  return 0;
}

// probe: partial sums over position groups, fixed-order sum, apply.
template <int K>
int launch_probe(ptycho_ctx* ctx, int mode, const float2* X, const float* w, bool want_den, bool apply) {
  ProbeArgs a{};
  a.O = ctx->O;
  a.nx = ctx->p.obj_nx;
  a.X = X;
  a.pos = ctx->pos;
  a.weights = w;
  a.J = ctx->p.J;
  a.M = ctx->p.M;
  a.G = ctx->S ? ctx->G_sub : ctx->G;
  if (ctx->blk.on) {  // this block's positions, added to the running sums
    a.J = ctx->blk.n;
    a.jlo = ctx->blk.j0;
    a.xoff = ctx->blk.j0;
    a.accumulate = ctx->blk.accumulate;
    a.G = std::min(ctx->G, ctx->blk.n);
  }
  if (ctx->S) {  // groups in bin order, one numerator per bin
    a.order = ctx->porder;
    a.goff = ctx->goff;
    a.bgrp = ctx->bgrp;
    a.nbins = ctx->S * ctx->S;
  }
  a.part_num = ctx->ppart;
  a.part_den = want_den ? ctx->ppart_den : nullptr;
  a.num = ctx->pnum;
  a.den = ctx->pden;
  a.blk_max = ctx->pblk_max;
  a.P = ctx->P;
  a.dP = ctx->dP;
  a.reg = (float)ctx->p.reg;
  a.beta = (float)ctx->p.lsqml_beta;
  const int MM = ctx->p.M * ctx->p.M;
  const int nblk = (MM + PROBE_NT - 1) / PROBE_NT;
  const double xb = (ctx->x16 && X == ctx->X ? 4.0 : 8.0) * a.J * K * (double)MM;
  if (X) {
    if (int r = launch(ctx, "probe_partial", xb, [&] {
          const bool h = ctx->x16 && X == ctx->X;  // FP16 residuals: two pixels per thread
          const int nbh = (MM / probe_px<__half2, K>() + PROBE_NT - 1) / PROBE_NT;
          if (ctx->S) {
            if (h) k_probe_partial<K, true, __half2><<<dim3(nbh, a.G), PROBE_NT, 0, ctx->st>>>(a);
            else k_probe_partial<K, true><<<dim3(nblk, a.G), PROBE_NT, 0, ctx->st>>>(a);
          } else {
            if (h) k_probe_partial<K, false, __half2><<<dim3(nbh, a.G), PROBE_NT, 0, ctx->st>>>(a);
            else k_probe_partial<K, false><<<dim3(nblk, a.G), PROBE_NT, 0, ctx->st>>>(a);
          }
        }))
      return r;
    ProbeArgs s = a;
    if (ctx->S) s.num = ctx->pbins;
    if (ctx->S && mode == PR_DM && want_den) s.bin_den = ctx->pbins_den;
    if (int r = launch(ctx, "probe_sum", 0.0, [&] { k_probe_sum<K><<<nblk, PROBE_NT, 0, ctx->st>>>(s); })) return r;
    if (ctx->S)  // adjoint shifts of the per-bin numerators, summed
      if (int r = launch_shift(ctx, false, ctx->pbins, ctx->pnum)) return r;
  }
  if (!apply) return 0;
  if (ctx->S && mode == PR_DM) return dm_probe_cg(ctx);
  switch (mode) {
    case PR_DM: return launch(ctx, "probe_apply", 0.0, [&] { k_probe_apply<K, PR_DM><<<nblk, PROBE_NT, 0, ctx->st>>>(a); });
    case PR_DIR: return launch(ctx, "probe_apply", 0.0, [&] { k_probe_apply<K, PR_DIR><<<nblk, PROBE_NT, 0, ctx->st>>>(a); });
    default: return launch(ctx, "probe_apply", 0.0, [&] { k_probe_apply<K, PR_UPD><<<nblk, PROBE_NT, 0, ctx->st>>>(a); });
  }
}

int probe_step(ptycho_ctx* ctx, int mode, const float2* X, const float* w, bool want_den, bool apply) {
  switch (ctx->p.K) {
    case 1: return launch_probe<1>(ctx, mode, X, w, want_den, apply);
    case 2: return launch_probe<2>(ctx, mode, X, w, want_den, apply);
    default: return launch_probe<3>(ctx, mode, X, w, want_den, apply);
  }
}

int steps_step(ptycho_ctx* ctx, bool upd) {
  if (upd && ctx->S)  // the probe direction as each position sees it
    if (int r = launch_shift(ctx, true, ctx->dP, ctx->dPt)) return r;
  StepArgs a{};
  a.O = ctx->O;
  a.dO = ctx->dO;
  a.nx = ctx->p.obj_nx;
  a.P = probe_view(ctx);
  a.dP = upd ? (ctx->S ? ctx->dPt : ctx->dP) : nullptr;
  a.pbin = bin_view(ctx);
  a.X = ctx->X;
  a.pos = ctx->pos;
  a.M = ctx->p.M;
  a.alpha_O = ctx->alphaO;
  a.alpha_P = ctx->alphaP;
  int J = ctx->p.J;
  if (ctx->blk.on) {
    a.j0 = ctx->blk.j0;
    a.xoff = ctx->blk.j0;
    J = ctx->blk.n;
  }
  a.nj = J;
  const bool h = ctx->x16;  // FP16 residuals (a.X is ctx->X)
  const double xb = (h ? 4.0 : 8.0) * J * ctx->p.K * (double)ctx->p.M * ctx->p.M;
  const bool sub = ctx->S != 0;
  auto go = [&](auto kern, unsigned grid) { kern<<<grid, STEP_NT, 0, ctx->st>>>(a); };
  switch (ctx->p.K) {
    case 1: return launch(ctx, "lsqml_steps", xb, [&] {
        if (sub) go(h ? k_lsqml_steps<1, true, __half2> : k_lsqml_steps<1, true>, J);
        else go(h ? k_lsqml_steps<1, false, __half2> : k_lsqml_steps<1, false>, J);
      });
    case 2: return launch(ctx, "lsqml_steps", xb, [&] {
        if (sub) go(h ? k_lsqml_steps<2, true, __half2> : k_lsqml_steps<2, true>, J);
        else go(h ? k_lsqml_steps<2, false, __half2> : k_lsqml_steps<2, false>, J);
      });
    default: return launch(ctx, "lsqml_steps", xb, [&] {
        if (sub) go(h ? k_lsqml_steps<3, true, __half2> : k_lsqml_steps<3, true>, J);
        else go(h ? k_lsqml_steps<3, false, __half2> : k_lsqml_steps<3, false>, J);
      });
  }
}

int ensure_work_buffers(ptycho_ctx* ctx) {
  const size_t MM = (size_t)ctx->p.M * ctx->p.M;
  const size_t K = ctx->p.K;
  const size_t xpos = ctx->B > 0 ? (size_t)std::min(ctx->B, ctx->p.J) : (size_t)ctx->p.J;
  if (int r = dalloc(ctx, &ctx->X, xpos * K * MM)) return r;
  if (ctx->B > 0)
    if (int r = dalloc(ctx, &ctx->objacc, (size_t)ctx->p.obj_ny * ctx->p.obj_nx)) return r;
  if (int r = dalloc(ctx, &ctx->dO, (size_t)ctx->p.obj_ny * ctx->p.obj_nx)) return r;
  if (int r = dalloc(ctx, &ctx->dP, K * MM)) return r;
  if (int r = dalloc(ctx, &ctx->ppart, (size_t)ctx->G_cap * K * MM)) return r;
  if (int r = dalloc(ctx, &ctx->ppart_den, (size_t)ctx->G_cap * MM)) return r;
  if (int r = dalloc(ctx, &ctx->pnum, K * MM)) return r;
  if (int r = dalloc(ctx, &ctx->pden, MM)) return r;
  if (int r = dalloc(ctx, &ctx->pblk_max, (MM + PROBE_NT - 1) / PROBE_NT)) return r;
  if (int r = dalloc(ctx, &ctx->alphaO, (size_t)ctx->p.J)) return r;
  if (int r = dalloc(ctx, &ctx->alphaP, (size_t)ctx->p.J)) return r;
  if (K > 1) {  // probe-mode orthogonalisation (allocated here: iterations may be graph-captured)
    if (int r = dalloc(ctx, &ctx->gram, K * K)) return r;
    if (int r = dalloc(ctx, &ctx->modeV, K * K)) return r;
  }
  return 0;
}

// ------------------------------------------------------------- algorithms
// DM: buffers and the initial exit waves psi = P_k O_j (outside any graph).
int dm_prepare(ptycho_ctx* ctx) {
  if (ctx->B > 0)
    return fail(ctx, PTYCHO_ERR_UNSUPPORTED, "DM keeps the exit waves of all positions (create with block_positions = 0)");
  if (int r = ensure_work_buffers(ctx)) return r;
  const int J = ctx->p.J, K = ctx->p.K, M = ctx->p.M;
  if (!ctx->psi_valid) {
    const size_t n_el = (size_t)J * K * M * M;
    if (int r = refresh_probe_table(ctx)) return r;
    if (int r = launch(ctx, "exit_waves", 8.0 * n_el, [&] {
          k_exit_waves<<<1184, 256, 0, ctx->st>>>(ctx->O, ctx->p.obj_nx, probe_view(ctx), bin_view(ctx), ctx->pos, J,
                                                   K, M, ctx->X);
        }))
      return r;
    ctx->psi_valid = true;
  }
  return 0;
}

// One DM iteration with the probe update on or off (all device work).
// Orthogonalise the probe modes (K > 1): Gram matrix, eigenvectors, mixing
// of the probe and, for DM, of the exit waves with the same unitary.
int ortho_step(ptycho_ctx* ctx, bool mix_psi) {
  const int K = ctx->p.K;
  if (K < 2) return 0;
  const int MM = ctx->p.M * ctx->p.M;
  if (int r = dalloc(ctx, &ctx->gram, (size_t)K * K)) return r;
  if (int r = dalloc(ctx, &ctx->modeV, (size_t)K * K)) return r;
  return launch(ctx, "probe_ortho", 8.0 * K * MM * (mix_psi ? 2.0 * ctx->p.J + 3.0 : 3.0), [&] {
    k_mode_gram<<<K * K, 256, 0, ctx->st>>>(ctx->P, K, MM, ctx->gram);
    k_mode_eig<<<1, 32, 0, ctx->st>>>(ctx->gram, K, ctx->modeV);
    k_mode_mix<<<(MM + 255) / 256, 256, 0, ctx->st>>>(ctx->P, 1, K, MM, ctx->modeV);
    if (mix_psi) k_mode_mix<<<1184, 256, 0, ctx->st>>>(ctx->X, (size_t)ctx->p.J, K, MM, ctx->modeV);
  });
}

int dm_step(ptycho_ctx* ctx, bool upd) {
  if (int r = refresh_probe_table(ctx)) return r;  // the probe may have changed since the last Fourier pass
  if (int r = obj_step(ctx, OBJ_STEP_DM, ctx->X, nullptr)) return r;
  if (upd)
    if (int r = probe_step(ctx, PR_DM, ctx->X, nullptr, true, true)) return r;
  if (int r = launch_fourier(ctx, FM_DM, ctx->X, nullptr, 0, ctx->p.J, "fourier_dm")) return r;
  if (upd && ctx->p.probe_ortho) return ortho_step(ctx, true);
  return 0;
}

int lsqml_prepare(ptycho_ctx* ctx) {
  if (int r = ensure_work_buffers(ctx)) return r;
  if (!ctx->st_side) {  // created here, outside any stream capture
    CK(cudaStreamCreateWithFlags(&ctx->st_side, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ctx->ev_join, cudaEventDisableTiming));
  }
  ctx->psi_valid = false;
  return 0;
}

// The sums of the object direction and of the probe direction read the same
// residual and the current (O, P) and write disjoint buffers: the probe's run
// on the second stream beside the object's (each alone is latency-limited
// below the HBM roofline).  Serial while profiling (clean per-kernel times)
// and with sub-pixel positions (the probe sums then use the shift tables).
int direction_sums(ptycho_ctx* ctx, bool upd) {
  const bool side = upd && ctx->st_side && !ctx->prof && ctx->S == 0;
  if (!side) {
    if (int r = obj_step(ctx, OBJ_STEP_DIR, ctx->X, nullptr)) return r;
    if (upd)
      if (int r = probe_step(ctx, PR_DIR, ctx->X, nullptr, true, true)) return r;
    return 0;
  }
  CK(cudaEventRecord(ctx->ev_fork, ctx->st));
  CK(cudaStreamWaitEvent(ctx->st_side, ctx->ev_fork, 0));
  cudaStream_t main = ctx->st;
  ctx->st = ctx->st_side;
  const int rp = probe_step(ctx, PR_DIR, ctx->X, nullptr, true, true);
  ctx->st = main;
  // joined whatever happened, so that a stream capture can end cleanly
  const cudaError_t e = cudaEventRecord(ctx->ev_join, ctx->st_side);
  const int ro = obj_step(ctx, OBJ_STEP_DIR, ctx->X, nullptr);
  const cudaError_t e2 = cudaStreamWaitEvent(ctx->st, ctx->ev_join, 0);
  if (rp) return rp;
  if (ro) return ro;
  if (e != cudaSuccess || e2 != cudaSuccess)
    return fail(ctx, PTYCHO_ERR_CUDA, "stream fork/join: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
  return 0;
}

// One LSQML iteration with the probe update on or off (all device work).
// LSQML residual into dst under the context's likelihood.
int launch_chi(ptycho_ctx* ctx, float2* dst) {
  const int mode = ctx->p.likelihood == PTYCHO_LIK_POISSON ? FM_CHIP : FM_CHI;
  return launch_fourier(ctx, mode, dst, nullptr, 0, ctx->p.J, "fourier_chi");
}

int lsqml_step_blocked(ptycho_ctx* ctx, bool upd);

int lsqml_step_impl(ptycho_ctx* ctx, bool upd);

// One LSQML iteration; with FP16 residual storage the residual passes of this
// iteration read and write ctx->X as __half2.
int lsqml_step(ptycho_ctx* ctx, bool upd) {
  ctx->x16 = ctx->p.residual_store == PTYCHO_R_F16;
  const int r = (ctx->B > 0 && ctx->B < ctx->p.J) ? lsqml_step_blocked(ctx, upd) : lsqml_step_impl(ctx, upd);
  ctx->x16 = false;
  return r;
}

int lsqml_step_impl(ptycho_ctx* ctx, bool upd) {
  if (int r = launch_chi(ctx, ctx->X)) return r;
  if (int r = direction_sums(ctx, upd)) return r;
  if (int r = steps_step(ctx, upd)) return r;
  if (upd)  // alpha_P-weighted probe numerator from the old object
    if (int r = probe_step(ctx, PR_UPD, ctx->X, ctx->alphaP, false, false)) return r;
  if (int r = obj_step(ctx, OBJ_UPD, ctx->X, ctx->alphaO)) return r;
  if (upd)
    if (int r = probe_step(ctx, PR_UPD, nullptr, nullptr, false, true)) return r;
  if (upd && ctx->p.probe_ortho) return ortho_step(ctx, false);
  return 0;
}

// LSQML with the residuals of B positions resident at a time: two Fourier
// passes per iteration.  Pass 1 sums the directions' numerators and
// denominators block by block; pass 2 recomputes each block's residual (the
// same (O, P), so the same chi) for its step sizes and the alpha-weighted
// update sums.  Same arithmetic as lsqml_step, sums grouped by block.
int lsqml_step_blocked(ptycho_ctx* ctx, bool upd) {
  const int J = ctx->p.J, B = ctx->B;
  const int mode = ctx->p.likelihood == PTYCHO_LIK_POISSON ? FM_CHIP : FM_CHI;
  int r = 0;
  for (int pass = 0; pass < 2 && !r; ++pass) {
    for (int j0 = 0; j0 < J && !r; j0 += B) {
      ctx->blk.on = true;
      ctx->blk.j0 = j0;
      ctx->blk.n = std::min(B, J - j0);
      ctx->blk.accumulate = j0 > 0;
      r = launch_fourier(ctx, mode, ctx->X, nullptr, j0, ctx->blk.n, "fourier_chi");
      if (!r && pass == 0) {
        r = obj_step(ctx, OBJ_STEP_DIR, ctx->X, nullptr);
        if (!r && upd) r = probe_step(ctx, PR_DIR, ctx->X, nullptr, true, false);
      } else if (!r) {
        r = steps_step(ctx, upd);
        if (!r && upd) r = probe_step(ctx, PR_UPD, ctx->X, ctx->alphaP, false, false);
        if (!r) r = obj_step(ctx, OBJ_STEP_ACC, ctx->X, ctx->alphaO);
      }
      ctx->blk = ptycho_ctx::Block{};
    }
    if (r) break;
    if (pass == 0) {
      r = obj_finish(ctx, OBJ_STEP_DIR);
      if (!r && upd) r = probe_step(ctx, PR_DIR, nullptr, nullptr, true, true);
    }
  }
  if (r) return r;
  const size_t n = (size_t)ctx->p.obj_ny * ctx->p.obj_nx;
  if (int rr = launch(ctx, "obj_update", n * 28.0, [&] {
        k_obj_apply_acc<<<1184, 256, 0, ctx->st>>>(ctx->O, ctx->objacc, ctx->denO, ctx->denO_max, (float)ctx->p.reg,
                                                    (float)ctx->p.lsqml_beta, n);
      }))
    return rr;
  if (upd)
    if (int rr = probe_step(ctx, PR_UPD, nullptr, nullptr, false, true)) return rr;
  if (upd && ctx->p.probe_ortho) return ortho_step(ctx, false);
  return 0;
}

int run_dm(ptycho_ctx* ctx, int n) {
  if (int r = dm_prepare(ctx)) return r;
  for (int it = 0; it < n; ++it) {
    if (int r = dm_step(ctx, ctx->t >= ctx->p.probe_start)) return r;
    ctx->t++;
  }
  return 0;
}

int run_lsqml(ptycho_ctx* ctx, int n) {
  if (int r = lsqml_prepare(ctx)) return r;
  for (int it = 0; it < n; ++it) {
    if (int r = lsqml_step(ctx, ctx->t >= ctx->p.probe_start)) return r;
    ctx->t++;
  }
  return 0;
}

// Visiting order of iterations t .. t + n - 1: identity for seed 0, else a
// Durstenfeld shuffle driven by SplitMix64(seed XOR t).
std::vector<int> epie_orders(const ptycho_ctx* ctx, int n) {
  const int J = ctx->p.J;
  std::vector<int> ord((size_t)n * J);
  for (int it = 0; it < n; ++it) {
    int* o = ord.data() + (size_t)it * J;
    for (int i = 0; i < J; ++i) o[i] = i;
    if (ctx->p.seed != 0) {
      SplitMix64 g{ctx->p.seed ^ (uint64_t)(ctx->t + it)};
      for (int i = J - 1; i > 0; --i) {
        const int r = (int)(g.next() % (uint64_t)(i + 1));
        std::swap(o[i], o[r]);
      }
    }
  }
  return ord;
}

// Sub-pixel ePIE: one position at a time through the general kernels.  The
// probe is carried in the frame of the position being visited (T_j P, in
// place in P): moving to the next position's frame is one shift by the
// difference of the two shifts (exact composition of Fourier shifts), the
// probe step is added in that frame, and the sweep ends with the shift back
// to the unshifted frame.  Per position: the frame shift (when the bin
// changes), the residual pass of the position, the maxima, the object and
// probe update.
template <int K>
int run_epie_subpixel_k(ptycho_ctx* ctx, int n) {
  const int J = ctx->p.J, M = ctx->p.M, MM = M * M, S = ctx->S, h = S / 2;
  const std::vector<int> ord = epie_orders(ctx, n);
  float2* D = ctx->cg_q;       // the position's residual
  float2* mx = ctx->ep_mx;     // partial (pmax, omax)
  int cy = h, cx = h;          // bins of the frame P is held in (h, h: unshifted)
  auto sweep = [&](int it) -> int {
    const bool upd = ctx->t + it >= ctx->p.probe_start;
    for (int s = 0; s < J; ++s) {
      const int j = ord[(size_t)it * J + s];
      const int by = ctx->bin_host[j] / S, bx = ctx->bin_host[j] % S;
      int nmx = EPS_MX;
      if (by != cy || bx != cx) {  // the frame change also gives the maxima
        if (int r = launch_frame_change<K>(ctx, by - cy + h, bx - cx + h, j, mx, &nmx)) return r;
        cy = by;
        cx = bx;
      } else if (int r = launch(ctx, "epie_max", 8.0 * (K + 1) * MM, [&] {
                   launch_k(ctx, k_epie_sub_max<K>, dim3(EPS_MX), dim3(EPS_NT), (const float2*)ctx->P,
                            (const float2*)ctx->O, ctx->p.obj_nx, (const int2*)ctx->pos, j, M, mx);
                 })) {
        return r;
      }
      ctx->f_P = ctx->P;
      ctx->f_xoff = j;
      ctx->f_ks = ctx->fks_one;
      int r = launch_fourier(ctx, FM_CHI, D, nullptr, j, 1, "fourier_epie");
      ctx->f_P = nullptr;
      ctx->f_xoff = -1;
      ctx->f_ks = nullptr;
      if (r) return r;
      if (int rr = launch(ctx, "epie_update", 8.0 * (3 * K + 2) * MM, [&] {
            launch_k(ctx, k_epie_sub_update<K>, dim3((MM + 255) / 256), dim3(256), ctx->O, ctx->p.obj_nx,
                     (const int2*)ctx->pos, j, M, ctx->P, (const float2*)D, (const float2*)mx, nmx,
                     (float)ctx->p.epie_alpha, (float)ctx->p.epie_beta, upd ? 1 : 0);
          }))
        return rr;
    }
    return 0;
  };
  for (int it = 0; it < n; ++it) {
    // chains of small dependent kernels: overlap each launch with its
    // predecessor's tail (not while profiling: events sit between launches)
    ctx->pdl = !ctx->prof;
    const int r = sweep(it);
    ctx->pdl = false;
    if (cy != h || cx != h) {  // back to the unshifted frame (also after an error)
      const int rb = launch_shift_one(ctx, h - cy + h, h - cx + h, ctx->P, ctx->P);
      cy = cx = h;
      if (!r && rb) return rb;
    }
    if (r) return r;
    if (ctx->t + it >= ctx->p.probe_start && ctx->p.probe_ortho && K > 1)
      if (int rr = ortho_step(ctx, false)) return rr;
  }
  ctx->t += n;
  ctx->psi_valid = false;
  return 0;
}

int run_epie(ptycho_ctx* ctx, int n) {
  if (ctx->S) {
    switch (ctx->p.K) {
      case 1: return run_epie_subpixel_k<1>(ctx, n);
      case 2: return run_epie_subpixel_k<2>(ctx, n);
      default: return run_epie_subpixel_k<3>(ctx, n);
    }
  }
  if (!ctx->epie_ok)
    return fail(ctx, PTYCHO_ERR_UNSUPPORTED, "ePIE kernel for M=%d K=%d cluster=%d exceeds shared memory; use a larger cluster",
                ctx->p.M, ctx->p.K, ctx->eks ? ctx->eks->C : ctx->C);
  const int J = ctx->p.J;
  const std::vector<int> ord = epie_orders(ctx, n);
  if ((size_t)ctx->order_cap < ord.size()) {
    dfree(ctx, ctx->order);
    if (int r = dalloc(ctx, &ctx->order, ord.size())) return r;
    ctx->order_cap = (int)ord.size();
  }
  CK(cudaMemcpyAsync(ctx->order, ord.data(), ord.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->st));
  EpieArgs a{};
  a.O = ctx->O;
  a.nx = ctx->p.obj_nx;
  a.P = ctx->P;
  a.pos = ctx->pos;
  a.amp = ctx->amp;
  a.amp_scale = ctx->amp_scale;
  a.istore = ctx->p.istore;
  a.tw = ctx->tw;
  a.order = ctx->order;
  a.J = J;
  a.n_iter = n;
  a.t0 = ctx->t;
  a.probe_start = ctx->p.probe_start;
  a.alpha = (float)ctx->p.epie_alpha;
  a.beta = (float)ctx->p.epie_beta;
  const KernelSet* ks = ctx->eks;
  auto sweep = [&](const EpieArgs& ea, int iters) {
    const double bytes = (double)iters * J * ctx->p.M * ctx->p.M * amp_bytes(ctx);
    return launch(ctx, "epie", bytes, [&] {
      cudaLaunchConfig_t cfg{};
      cfg.gridDim = dim3((unsigned)ks->C);
      cfg.blockDim = dim3((unsigned)(ctx->epie2 ? ks->NT2 : ks->NT_epie));
      cfg.dynamicSmemBytes = ctx->epie2 ? ks->smem_epie2 : ks->smem_epie;
      cfg.stream = ctx->st;
      cudaLaunchAttribute attr[1];
      if (ks->C > 1) {
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = ks->C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
      }
      if (ctx->epie2) {
        Epie2Args e2{};
        e2.O = ea.O;
        e2.nx = ea.nx;
        e2.P = ea.P;
        e2.pos = ea.pos;
        e2.amp = ea.amp;
        e2.amp_scale = ea.amp_scale;
        e2.istore = ea.istore;
        e2.tw2 = ctx->tw2;
        e2.order = ea.order;
        e2.J = ea.J;
        e2.n_iter = ea.n_iter;
        e2.t0 = ea.t0;
        e2.probe_start = ea.probe_start;
        e2.alpha = ea.alpha;
        e2.beta = ea.beta;
        e2.err_flag = ctx->err_flag;
        cudaLaunchKernelEx(&cfg, ks->epie2, e2);
      } else {
        cudaLaunchKernelEx(&cfg, ks->epie, ea);
      }
    });
  };
  int r = 0;
  if (ctx->p.probe_ortho && ctx->p.K > 1) {
    // one sweep per launch, the modes orthogonalised after each sweep that
    // updated the probe
    for (int it = 0; it < n && !r; ++it) {
      EpieArgs e1 = a;
      e1.order = ctx->order + (size_t)it * J;
      e1.n_iter = 1;
      e1.t0 = ctx->t + it;
      r = sweep(e1, 1);
      if (!r && ctx->t + it >= ctx->p.probe_start) r = ortho_step(ctx, false);
    }
  } else {
    r = sweep(a, n);
  }
  if (r) return r;
  // the host order buffer must outlive the async copy
  CK(cudaStreamSynchronize(ctx->st));
  ctx->t += n;
  ctx->psi_valid = false;
  return 0;
}

// Sub-pixel positions: the probe-sum groups in bin order.  Bin b's n_b
// positions (ascending index) are cut into max(1, ceil(n_b G / J)) groups, so
// there are at most G + S^2 of them; empty bins get none.
int build_subpixel_groups(ptycho_ctx* ctx, const std::vector<unsigned short>& bin) {
  const int J = ctx->p.J, nb = ctx->S * ctx->S;
  std::vector<int> start(nb + 1, 0);
  for (int j = 0; j < J; ++j) start[bin[j] + 1]++;
  for (int b = 0; b < nb; ++b) start[b + 1] += start[b];
  std::vector<int> order(J), fill(start.begin(), start.end() - 1);
  for (int j = 0; j < J; ++j) order[fill[bin[j]]++] = j;
  std::vector<int> goff, bgrp(nb + 1);
  for (int b = 0; b < nb; ++b) {
    bgrp[b] = (int)goff.size();
    const int n = start[b + 1] - start[b];
    if (n == 0) continue;
    int g = (int)(((long long)n * ctx->G + J - 1) / J);
    g = std::max(1, std::min(g, n));
    for (int i = 0; i < g; ++i) goff.push_back(start[b] + (int)((long long)n * i / g));
  }
  bgrp[nb] = (int)goff.size();
  goff.push_back(J);
  const int G = (int)goff.size() - 1;
  if (G > ctx->G_cap) return fail(ctx, PTYCHO_ERR_ARG, "internal: %d probe-sum groups exceed %d", G, ctx->G_cap);
  CK(cudaMemcpyAsync(ctx->porder, order.data(), J * sizeof(int), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->goff, goff.data(), goff.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->bgrp, bgrp.data(), bgrp.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));  // the host vectors end with this call
  ctx->G_sub = G;
  return 0;
}

int set_positions_impl(ptycho_ctx* ctx, const float* positions) {
  if (!positions) return fail(ctx, PTYCHO_ERR_ARG, "positions is NULL");
  const int J = ctx->p.J, M = ctx->p.M, ny = ctx->p.obj_ny, nx = ctx->p.obj_nx, S = ctx->S;
  std::vector<int2> pos(J);
  std::vector<unsigned short> bin(S ? J : 0);
  for (int j = 0; j < J; ++j) {
    const float fy = positions[2 * j], fx = positions[2 * j + 1];
    if (!std::isfinite(fy) || !std::isfinite(fx))
      return fail(ctx, PTYCHO_ERR_NONFINITE, "position %d is not finite", j);
    double y, x;
    if (S) {
      // quantised to 1/S pixel (half to even), corner floor((q + S/2) / S),
      // shift bin q - S corner + S/2 in [0, S)
      const double qy = std::nearbyint((double)S * fy), qx = std::nearbyint((double)S * fx);
      y = std::floor((qy + S / 2) / S);
      x = std::floor((qx + S / 2) / S);
      if (std::fabs(qy) > 1e9 || std::fabs(qx) > 1e9)
        return fail(ctx, PTYCHO_ERR_BOUNDS, "position %d is far outside the object", j);
      const int by = (int)(qy - S * y) + S / 2, bx = (int)(qx - S * x) + S / 2;
      bin[j] = (unsigned short)(by * S + bx);
    } else {
      y = std::nearbyint((double)fy);
      x = std::nearbyint((double)fx);
    }
    if (y < 0 || x < 0 || y + M > ny || x + M > nx)
      return fail(ctx, PTYCHO_ERR_BOUNDS, "patch %d at (%g, %g) falls outside the %dx%d object", j, y, x, ny, nx);
    pos[j] = make_int2((int)y, (int)x);
  }
  if (S) {
    const size_t tab = (size_t)S * S * ctx->p.K * M * M;
    if (int r = dalloc(ctx, &ctx->pbin, (size_t)J)) return r;
    if (int r = dalloc(ctx, &ctx->Pt, tab)) return r;
    if (int r = dalloc(ctx, &ctx->dPt, tab)) return r;
    if (int r = dalloc(ctx, &ctx->pbins, tab)) return r;
    if (int r = dalloc(ctx, &ctx->stmp, (size_t)S * ctx->p.K * M * M)) return r;
    if (int r = dalloc(ctx, &ctx->porder, (size_t)J)) return r;
    if (int r = dalloc(ctx, &ctx->goff, (size_t)ctx->G_cap + 1)) return r;
    if (int r = dalloc(ctx, &ctx->bgrp, (size_t)S * S + 1)) return r;
    const size_t KMM = (size_t)ctx->p.K * M * M;
    if (int r = dalloc(ctx, &ctx->pbins_den, (size_t)S * S * M * M)) return r;
    if (int r = dalloc(ctx, &ctx->cg_r, KMM)) return r;
    if (int r = dalloc(ctx, &ctx->cg_p, KMM)) return r;
    if (int r = dalloc(ctx, &ctx->cg_q, KMM)) return r;
    if (int r = dalloc(ctx, &ctx->cg_part, 3 * ((KMM + CG_NT - 1) / CG_NT))) return r;
    if (int r = dalloc(ctx, &ctx->pos_corr, (size_t)J)) return r;
    if (int r = dalloc(ctx, &ctx->ep_mx, (size_t)EPS_MX_CAP)) return r;
    CK(cudaMemcpyAsync(ctx->pbin, bin.data(), J * sizeof(unsigned short), cudaMemcpyHostToDevice, ctx->st));
    ctx->bin_host = bin;
    if (int r = build_subpixel_groups(ctx, bin)) return r;
  }
  // CSR lists of positions per object tile, ascending position index
  std::vector<int> cnt(ctx->n_tiles + 1, 0);
  for (int j = 0; j < J; ++j) {
    const int t0y = pos[j].x / TILE_Y, t1y = (pos[j].x + M - 1) / TILE_Y;
    const int t0x = pos[j].y / TILE_X, t1x = (pos[j].y + M - 1) / TILE_X;
    for (int ty = t0y; ty <= t1y; ++ty)
      for (int tx = t0x; tx <= t1x; ++tx) cnt[ty * ctx->ntx + tx + 1]++;
  }
  for (int i = 0; i < ctx->n_tiles; ++i) cnt[i + 1] += cnt[i];
  std::vector<int> list(cnt[ctx->n_tiles]);
  std::vector<int> fill(cnt.begin(), cnt.end() - 1);
  for (int j = 0; j < J; ++j) {
    const int t0y = pos[j].x / TILE_Y, t1y = (pos[j].x + M - 1) / TILE_Y;
    const int t0x = pos[j].y / TILE_X, t1x = (pos[j].y + M - 1) / TILE_X;
    for (int ty = t0y; ty <= t1y; ++ty)
      for (int tx = t0x; tx <= t1x; ++tx) list[fill[ty * ctx->ntx + tx]++] = j;
  }
  // the tile lists keep their allocation while they fit (a free would wait
  // for the whole device, other contexts' work included); the uploads are
  // ordered on the context's stream after its own earlier kernels, which
  // read the lists they replace
  if (list.size() + 1 > ctx->tile_list_cap) {
    dfree(ctx, ctx->tile_list);
    ctx->tile_list_cap = 0;
    if (int r = dalloc(ctx, &ctx->tile_list, list.size() + 1)) return r;
    ctx->tile_list_cap = list.size() + 1;
  }
  CK(cudaMemcpyAsync(ctx->pos, pos.data(), J * sizeof(int2), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->tile_ptr, cnt.data(), cnt.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->st));
  CK(cudaMemcpyAsync(ctx->tile_list, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice, ctx->st));
  // the sources are host vectors of this call: wait until the copies have
  // consumed them (a pageable copy may return before it has)
  CK(cudaStreamSynchronize(ctx->st));
  ctx->pos_host = pos;
  ctx->pos_f.assign(positions, positions + 2 * (size_t)J);
  ctx->have_pos = true;
  ctx->psi_valid = false;
  return 0;
}

int copy_out(ptycho_ctx* ctx, float* out, const void* src, size_t bytes, int on_device) {
  if (!out) return fail(ctx, PTYCHO_ERR_ARG, "output pointer is NULL");
  CK(cudaMemcpyAsync(out, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  return 0;
}

}  // namespace

// ---------------------------------------------------------------------------
// Allocation-free Fourier error.  Its scratch is one file-scope device array
// that every GPU loading this library holds until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr int NOALLOC_MAX_J = 16384;   // positions per call
constexpr int NOALLOC_MAX_M = 256;
constexpr int NOALLOC_MAX_C = 16;  // largest compiled cluster size
// layout: [twiddles M_max float2][flag int, pad][err_out double2][positions int2 x J_max]
//         [per-CTA error partials double2 x J_max * C_max]
constexpr size_t NA_TW = 0;
constexpr size_t NA_FLAG = NA_TW + NOALLOC_MAX_M * sizeof(float2);
constexpr size_t NA_OUT = NA_FLAG + 256;
constexpr size_t NA_POS = NA_OUT + 256;
constexpr size_t NA_PART = NA_POS + (size_t)NOALLOC_MAX_J * sizeof(int2);
constexpr size_t NA_BYTES = NA_PART + (size_t)NOALLOC_MAX_J * NOALLOC_MAX_C * sizeof(double2);

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// With the caller's device current: the device address of the scratch
// array (its host-side name is only a stand-in).  Looked up on every call --
// a lookup allocates nothing -- so that no address outlives the module it
// belongs to (a device reset reloads the module).
int noalloc_scratch(unsigned char** out) {
  void* ptr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
  if (e != cudaSuccess || !ptr)
    return fail(nullptr, PTYCHO_ERR_CUDA, "cudaGetSymbolAddress of the scratch array: %s", cudaGetErrorString(e));
  *out = (unsigned char*)ptr;
  return 0;
}

// A caller's input pointer must be device (or managed) memory of the current
// device: a host pointer reaching the kernel would fault (or, where the GPU
// can reach host memory, read the wrong memory).
int noalloc_check_device_ptr(const void* p, int dev, const char* what) {
  cudaPointerAttributes at{};
  const cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(nullptr, PTYCHO_ERR_ARG, "%s: not a CUDA pointer (%s)", what, cudaGetErrorString(e));
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    return fail(nullptr, PTYCHO_ERR_ARG, "%s is not device memory", what);
  if (at.type == cudaMemoryTypeDevice && at.device != dev)
    return fail(nullptr, PTYCHO_ERR_ARG, "%s lives on device %d, the current device is %d", what, at.device, dev);
  return 0;
}

}  // namespace

extern "C" int ptycho_fourier_error_noalloc(const float* object, int obj_ny, int obj_nx, const float* probe, int M,
                                            int K, const float* positions, int J, const float* amplitudes,
                                            double* out, void* stream) {
  if (!object || !probe || !positions || !amplitudes || !out)
    return fail(nullptr, PTYCHO_ERR_ARG, "NULL argument");
  if (M < 2 || K < 1 || J < 1 || obj_ny < M || obj_nx < M)
    return fail(nullptr, PTYCHO_ERR_ARG, "bad sizes M=%d K=%d J=%d object %dx%d", M, K, J, obj_ny, obj_nx);
  if (J > NOALLOC_MAX_J || M > NOALLOC_MAX_M)
    return fail(nullptr, PTYCHO_ERR_ARG,
                "J=%d, M=%d exceed the fixed scratch of the allocation-free call (at most J=%d, M=%d)", J, M,
                NOALLOC_MAX_J, NOALLOC_MAX_M);
  // the kernel reads amplitudes with 16-byte bulk operations and the object
  // and probe as 8-byte complex values
  if ((uintptr_t)amplitudes % 16 != 0) return fail(nullptr, PTYCHO_ERR_ARG, "amplitudes are not 16-byte aligned");
  if ((uintptr_t)object % 8 != 0 || (uintptr_t)probe % 8 != 0)
    return fail(nullptr, PTYCHO_ERR_ARG, "object and probe must be 8-byte aligned");
  const int C = default_cluster(M, K);
  const KernelSet* ks = C ? find_set(M, K, C) : nullptr;
  if (!ks) return fail(nullptr, PTYCHO_ERR_UNSUPPORTED, "no kernel compiled for M=%d K=%d", M, K);
  if (C > NOALLOC_MAX_C) return fail(nullptr, PTYCHO_ERR_UNSUPPORTED, "cluster size %d exceeds the scratch layout", C);
  // positions: round half-to-even, check bounds, stage in one host buffer
  std::vector<int2> hpos((size_t)J);
  for (int j = 0; j < J; ++j) {
    const float fy = positions[2 * j], fx = positions[2 * j + 1];
    if (!std::isfinite(fy) || !std::isfinite(fx)) return fail(nullptr, PTYCHO_ERR_NONFINITE, "position %d is not finite", j);
    const double y = std::nearbyint((double)fy), x = std::nearbyint((double)fx);
    if (y < 0 || x < 0 || y + M > obj_ny || x + M > obj_nx)
      return fail(nullptr, PTYCHO_ERR_BOUNDS, "patch %d at (%g, %g) falls outside the %dx%d object", j, y, x, obj_ny,
                  obj_nx);
    hpos[j] = make_int2((int)y, (int)x);
  }
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(nullptr, PTYCHO_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (int r = noalloc_check_device_ptr(object, dev, "object")) return r;
  if (int r = noalloc_check_device_ptr(probe, dev, "probe")) return r;
  if (int r = noalloc_check_device_ptr(amplitudes, dev, "amplitudes")) return r;
  unsigned char* sc = nullptr;
  if (int r = noalloc_scratch(&sc)) return r;
  cudaStream_t st = (cudaStream_t)stream;
  int2* pos = (int2*)(sc + NA_POS);
  e = cudaMemcpyAsync(pos, hpos.data(), (size_t)J * sizeof(int2), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail(nullptr, PTYCHO_ERR_CUDA, "position upload: %s", cudaGetErrorString(e));
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess && ks->smem_fourier > (size_t)optin)
    return fail(nullptr, PTYCHO_ERR_UNSUPPORTED, "Fourier kernel needs more shared memory than the device offers");
  if (e == cudaSuccess) e = set_fourier_attributes(ks);
  if (e == cudaSuccess) e = cudaMemsetAsync(sc + NA_FLAG, 0, sizeof(int), st);  // the only state that must start at 0
  if (e != cudaSuccess) return fail(nullptr, PTYCHO_ERR_CUDA, "setup: %s", cudaGetErrorString(e));
  k_twiddle2<<<(M + 255) / 256, 256, 0, st>>>((float2*)(sc + NA_TW), M, M / radix1(M));
  Fourier2Args a{};
  a.O = (const float2*)object;
  a.nx = obj_nx;
  a.P = (const float2*)probe;
  a.pos = pos;
  a.amp = amplitudes;
  a.istore = PTYCHO_I_F32;
  a.err_part = (double2*)(sc + NA_PART);
  a.tw2 = (const float2*)(sc + NA_TW);
  a.err_flag = (int*)(sc + NA_FLAG);
  a.wait_limit = 1 << 20;
  a.nj = J;
  a.mode = FM_ERR;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3((unsigned)(ks->C * J));
  cfg.blockDim = dim3((unsigned)ks->NT2);
  cfg.dynamicSmemBytes = ks->smem_fourier;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  if (ks->C > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ks->C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  cudaLaunchKernelEx(&cfg, ks->fourier, a);
  k_err_final<<<1, 1024, 0, st>>>((const double2*)(sc + NA_PART), J * ks->C, (double2*)(sc + NA_OUT));
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(nullptr, PTYCHO_ERR_CUDA, "launch: %s", cudaGetErrorString(e));
  struct {
    double2 v;
    int flag;
  } h{};
  e = cudaMemcpyAsync(&h.v, sc + NA_OUT, sizeof(double2), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h.flag, sc + NA_FLAG, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(nullptr, PTYCHO_ERR_CUDA, "fourier_error_noalloc: %s", cudaGetErrorString(e));
  if (h.flag) return fail(nullptr, PTYCHO_ERR_TIMEOUT, "a bounded device wait gave up (bulk copy did not complete)");
  const double E = h.v.y > 0 ? h.v.x / h.v.y : 0.0;
  *out = E;
  if (!std::isfinite(E)) return fail(nullptr, PTYCHO_ERR_DIVERGED, "Fourier error is not finite");
  return PTYCHO_OK;
}

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------
extern "C" {

void ptycho_default_params(ptycho_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof *p);
  p->istore = PTYCHO_I_F32;
  p->probe_start = 0;
  p->epie_alpha = 1.0;
  p->epie_beta = 1.0;
  p->lsqml_beta = 0.9;
  p->reg = 1e-3;
  p->seed = 0;
  p->stream = nullptr;
  p->cluster = 0;
  p->likelihood = PTYCHO_LIK_AMPLITUDE;
  p->probe_ortho = 0;
  p->subpixel = 0;
  p->block_positions = 0;
}

static int create_impl(ptycho_ctx** out, const ptycho_params* p);

int ptycho_create(ptycho_ctx** out, const ptycho_params* p) {
  if (p && p->fft_engine == PTYCHO_FFT_AUTO) {  // the measured faster engine for (M, K)
    ptycho_params q = *p;
    int eng = PTYCHO_FFT_REGISTER, C = 0;
    if (q.M >= 2 && q.K >= 1 && ptycho_autotune_engine(q.M, q.K, &eng, &C, nullptr) == PTYCHO_OK) {
      q.fft_engine = eng;
      if (q.cluster < 0) q.cluster = C;
    } else {
      q.fft_engine = PTYCHO_FFT_REGISTER;
    }
    return create_impl(out, &q);
  }
  return create_impl(out, p);
}

static int create_impl(ptycho_ctx** out, const ptycho_params* p) {
  ptycho_ctx* ctx = nullptr;
  if (!out || !p) return fail(nullptr, PTYCHO_ERR_ARG, "NULL argument");
  *out = nullptr;
  if (p->M < 2 || p->K < 1 || p->J < 1 || p->obj_ny < p->M || p->obj_nx < p->M)
    return fail(nullptr, PTYCHO_ERR_ARG, "bad sizes M=%d K=%d J=%d object %dx%d", p->M, p->K, p->J, p->obj_ny,
                p->obj_nx);
  if (p->K > 3) return fail(nullptr, PTYCHO_ERR_UNSUPPORTED, "K=%d modes: at most 3 are compiled in", p->K);
  if (p->istore < 0 || p->istore > 2) return fail(nullptr, PTYCHO_ERR_ARG, "istore=%d", p->istore);
  if (p->likelihood != PTYCHO_LIK_AMPLITUDE && p->likelihood != PTYCHO_LIK_POISSON)
    return fail(nullptr, PTYCHO_ERR_ARG, "likelihood=%d", p->likelihood);
  if (p->probe_ortho != 0 && p->probe_ortho != 1) return fail(nullptr, PTYCHO_ERR_ARG, "probe_ortho=%d", p->probe_ortho);
  if (p->K > MODE_KMAX) return fail(nullptr, PTYCHO_ERR_UNSUPPORTED, "K=%d probe modes (at most %d)", p->K, MODE_KMAX);
  if (p->subpixel != 0 && p->subpixel != 2 && p->subpixel != 4 && p->subpixel != 8 && p->subpixel != 16)
    return fail(nullptr, PTYCHO_ERR_ARG, "subpixel=%d (0, 2, 4, 8 or 16)", p->subpixel);
  if (p->block_positions < 0) return fail(nullptr, PTYCHO_ERR_ARG, "block_positions=%d", p->block_positions);
  if (p->block_positions > 0 && p->subpixel > 0)
    return fail(nullptr, PTYCHO_ERR_UNSUPPORTED, "position blocks with sub-pixel positions are not supported");
  if (!(p->reg >= 0.0) || !std::isfinite(p->epie_alpha) || !std::isfinite(p->epie_beta) ||
      !std::isfinite(p->lsqml_beta))
    return fail(nullptr, PTYCHO_ERR_ARG, "non-finite or negative step parameter");
  if (p->residual_store != PTYCHO_R_F32 && p->residual_store != PTYCHO_R_F16)
    return fail(nullptr, PTYCHO_ERR_ARG, "residual_store=%d", p->residual_store);
  if (p->fft_engine != PTYCHO_FFT_REGISTER && p->fft_engine != PTYCHO_DFT_TENSOR_BF16X3)
    return fail(nullptr, PTYCHO_ERR_ARG, "fft_engine=%d", p->fft_engine);
  if (p->fft_engine == PTYCHO_DFT_TENSOR_BF16X3 && (p->M != 64 || p->K != 1))
    return fail(nullptr, PTYCHO_ERR_UNSUPPORTED, "the tensor-core DFT is compiled for M=64, K=1 (got M=%d K=%d)",
                p->M, p->K);
  int C = p->cluster > 0 ? p->cluster : default_cluster(p->M, p->K);
  if (p->cluster < 0) {  // autotuned: the fastest compiled cluster size for (M, K)
    int best = 0;
    if (ptycho_autotune(p->M, p->K, &best, nullptr) == PTYCHO_OK) C = best;
  }
  const KernelSet* ks = find_set(p->M, p->K, C);
  if (!ks)
    return fail(nullptr, PTYCHO_ERR_UNSUPPORTED, "no kernel compiled for M=%d K=%d cluster=%d", p->M, p->K, C);
  if ((long long)p->J * p->M * p->M > (1LL << 40)) return fail(nullptr, PTYCHO_ERR_ARG, "J*M*M too large");
  ctx = new ptycho_ctx();
  ctx->p = *p;
  ctx->st = (cudaStream_t)p->stream;
  ctx->ks = ks;
  ctx->C = C;
  ctx->ntx = (p->obj_nx + TILE_X - 1) / TILE_X;
  ctx->nty = (p->obj_ny + TILE_Y - 1) / TILE_Y;
  ctx->n_tiles = ctx->ntx * ctx->nty;
  {
    const int MM = p->M * p->M;
    const int nblk = (MM + PROBE_NT - 1) / PROBE_NT;
    int G = (16 * 148 + nblk - 1) / nblk;  // ~16 CTAs per SM of position groups
    if (G > p->J) G = p->J;
    if (G < 1) G = 1;
    ctx->G = G;
    ctx->S = p->subpixel;
    ctx->G_cap = G + ctx->S * ctx->S;
    ctx->B = p->block_positions < p->J ? p->block_positions : 0;
  }
  int r = 0;
  const size_t obj = (size_t)p->obj_ny * p->obj_nx;
  const size_t MM = (size_t)p->M * p->M;
  if (!r) r = dalloc(ctx, &ctx->O, obj);
  if (!r) r = dalloc(ctx, &ctx->P, (size_t)p->K * MM);
  if (!r) r = dalloc(ctx, &ctx->tw, (size_t)p->M);
  if (!r) r = dalloc(ctx, &ctx->tw2, (size_t)p->M);
  if (!r) r = dalloc(ctx, &ctx->err_flag, 1);
  if (!r) r = dalloc(ctx, &ctx->pos, (size_t)p->J);
  if (!r) r = dalloc(ctx, &ctx->denO, obj);
  if (!r) r = dalloc(ctx, &ctx->tile_max, (size_t)ctx->n_tiles);
  if (!r) r = dalloc(ctx, &ctx->denO_max, 1);
  if (!r) r = dalloc(ctx, &ctx->tile_ptr, (size_t)ctx->n_tiles + 1);
  if (!r) r = dalloc(ctx, &ctx->err_part, (size_t)p->J * C);
  if (!r) r = dalloc(ctx, &ctx->err_out, 1);
  if (!r) r = dalloc(ctx, &ctx->flag, 1);
  if (!r) {
    if (p->istore == PTYCHO_I_F32) r = dalloc(ctx, (float**)&ctx->amp, (size_t)p->J * MM);
    else r = dalloc(ctx, (__half**)&ctx->amp, (size_t)p->J * MM);
  }
  if (!r) r = dalloc(ctx, &ctx->amp_scale, (size_t)p->J);
  if (!r && p->fft_engine == PTYCHO_DFT_TENSOR_BF16X3)
    r = dalloc(ctx, &ctx->dftm, 2 * TC64_AMAT);
  if (r) {
    g_create_error = ctx->err;
    ptycho_destroy(ctx);
    return r;
  }
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess && ks->smem_fourier > (size_t)optin) {
    g_create_error = "Fourier kernel needs more shared memory than the device offers";
    ptycho_destroy(ctx);
    return PTYCHO_ERR_UNSUPPORTED;
  }
  if (e == cudaSuccess) e = set_fourier_attributes(ks);
  if (e == cudaSuccess) ctx->eks = epie_set(p, ks, optin);
  const KernelSet* eks = ctx->eks;
  // one position at a time (sub-pixel ePIE) the largest cluster is the
  // shortest chain: the ePIE set's Fourier kernels where they fit
  ctx->fks_one = ks;
  if (e == cudaSuccess && eks && eks != ks && eks->C > ks->C && eks->smem_fourier <= (size_t)optin &&
      eks->smem_spec <= (size_t)optin && set_fourier_attributes(eks) == cudaSuccess)
    ctx->fks_one = eks;
  cudaGetLastError();
  // the register-resident sweep where it is compiled and fits, else the
  // shared-memory-pass one
  ctx->epie2 = e == cudaSuccess && eks->epie2 != nullptr && eks->smem_epie2 <= (size_t)optin;
  if (ctx->epie2) {
    if (eks->C > 8) e = cudaFuncSetAttribute(eks->epie2, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(eks->epie2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)eks->smem_epie2);
    ctx->epie_ok = e == cudaSuccess;
  } else {
    if (e == cudaSuccess && eks->C > 8 && eks->epie)
      e = cudaFuncSetAttribute(eks->epie, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    ctx->epie_ok = e == cudaSuccess && eks->epie != nullptr && eks->smem_epie <= (size_t)optin;
    if (ctx->epie_ok)
      e = cudaFuncSetAttribute(eks->epie, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)eks->smem_epie);
  }
  if (e == cudaSuccess && p->fft_engine == PTYCHO_DFT_TENSOR_BF16X3) {
    for (int mode : {FM_DM, FM_CHI, FM_CHIP, FM_ERR, FM_SIM})
      for (int ist = 0; ist < 3 && e == cudaSuccess; ++ist)
        e = cudaFuncSetAttribute(tc64_fourier(mode, ist), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC64_SMEM);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) tc64_build_matrix(ctx->dftm, ctx->st);
  }
  if (e == cudaSuccess) {
    k_twiddle<<<(p->M + 255) / 256, 256, 0, ctx->st>>>(ctx->tw, p->M);
    k_twiddle2<<<(p->M + 255) / 256, 256, 0, ctx->st>>>(ctx->tw2, p->M, p->M / radix1(p->M));
    cudaMemsetAsync(ctx->err_flag, 0, sizeof(int), ctx->st);
    k_fill_c<<<256, 256, 0, ctx->st>>>(ctx->O, obj, make_float2(1.f, 0.f));
    k_fill_c<<<256, 256, 0, ctx->st>>>(ctx->P, (size_t)p->K * MM, make_float2(0.f, 0.f));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
  if (e != cudaSuccess) {
    g_create_error = std::string("device setup failed: ") + cudaGetErrorString(e);
    ptycho_destroy(ctx);
    return PTYCHO_ERR_CUDA;
  }
  *out = ctx;
  return PTYCHO_OK;
}

int ptycho_set_positions(ptycho_ctx* ctx, const float* positions) {
  if (!ctx) return PTYCHO_ERR_ARG;
  return set_positions_impl(ctx, positions);
}

// sqrt(I) in FFT order (and the 16-bit scales) for frames [j0, j0 + nj) read
// from src (frame j0 at src[0]).
static int prepare_amp(ptycho_ctx* ctx, const float* src, int j0, int nj) {
  const int M = ctx->p.M;
  const size_t MM = (size_t)M * M;
  const bool vec = ((uintptr_t)src & 15) == 0;
  const dim3 grid((unsigned)M, (unsigned)std::min(nj, 65535));
  const unsigned nt = (unsigned)std::min(256, std::max(32, M / 4));
  if (ctx->p.istore == PTYCHO_I_F32)
    return launch(ctx, "prepare_amp", 8.0 * nj * MM, [&] {
      float* dst = (float*)ctx->amp + (size_t)j0 * MM;
      if (vec) k_amp_f32<4><<<grid, nt, 0, ctx->st>>>(src, nj, M, dst, ctx->flag);
      else k_amp_f32<1><<<grid, nt, 0, ctx->st>>>(src, nj, M, dst, ctx->flag);
    });
  if (int rc = launch(ctx, "frame_max", 4.0 * nj * MM,
                      [&] { k_frame_max<<<nj, 256, 0, ctx->st>>>(src, M, ctx->amp_scale + j0, ctx->flag); }))
    return rc;
  if (ctx->p.istore == PTYCHO_I_F16)
    return launch(ctx, "prepare_amp", 6.0 * nj * MM, [&] {
      __half* dst = (__half*)ctx->amp + (size_t)j0 * MM;
      if (vec) k_amp_q16<__half, 4><<<grid, nt, 0, ctx->st>>>(src, nj, M, ctx->amp_scale + j0, dst);
      else k_amp_q16<__half, 1><<<grid, nt, 0, ctx->st>>>(src, nj, M, ctx->amp_scale + j0, dst);
    });
  return launch(ctx, "prepare_amp", 6.0 * nj * MM, [&] {
    __nv_bfloat16* dst = (__nv_bfloat16*)ctx->amp + (size_t)j0 * MM;
    if (vec) k_amp_q16<__nv_bfloat16, 4><<<grid, nt, 0, ctx->st>>>(src, nj, M, ctx->amp_scale + j0, dst);
    else k_amp_q16<__nv_bfloat16, 1><<<grid, nt, 0, ctx->st>>>(src, nj, M, ctx->amp_scale + j0, dst);
  });
}

}  // extern "C"

namespace {

// Frames from host memory in chunks of `chunk` frames, double-buffered on the
// copy stream: the upload of one chunk overlaps the processing of the
// previous one; process(dev, j0, nj) reads the chunk's nj <= chunk frames at
// dev on ctx->st.
template <class Fn>
int upload_chunks(ptycho_ctx* ctx, const unsigned char* host, size_t frame_bytes, int J, int chunk, Fn&& process) {
  if (int r = ensure_stage(ctx, 2 * (size_t)chunk * frame_bytes)) return r;
  cudaEvent_t ready = get_event(ctx);
  CK(cudaEventRecord(ready, ctx->st));  // earlier users of the stage are done
  CK(cudaStreamWaitEvent(ctx->st_copy, ready, 0));
  ctx->ev_pool.push_back(ready);
  int rc = 0;
  for (int j0 = 0, c = 0; j0 < J && !rc; j0 += chunk, ++c) {
    const int nj = std::min(chunk, J - j0), h = c & 1;
    unsigned char* half = reinterpret_cast<unsigned char*>(ctx->stage) + (size_t)h * chunk * frame_bytes;
    if (c >= 2) CK(cudaStreamWaitEvent(ctx->st_copy, ctx->ev_used[h], 0));
    cudaError_t e = cudaMemcpyAsync(half, host + (size_t)j0 * frame_bytes, (size_t)nj * frame_bytes,
                                    cudaMemcpyHostToDevice, ctx->st_copy);
    if (e != cudaSuccess) return fail(ctx, PTYCHO_ERR_CUDA, "frame upload: %s", cudaGetErrorString(e));
    CK(cudaEventRecord(ctx->ev_copied[h], ctx->st_copy));
    CK(cudaStreamWaitEvent(ctx->st, ctx->ev_copied[h], 0));
    rc = process(half, j0, nj);
    CK(cudaEventRecord(ctx->ev_used[h], ctx->st));
  }
  return rc;
}

// Read the NaN/Inf flag of the uploads and mark the data present.
int finish_set_data(ptycho_ctx* ctx, int rc, const char* what) {
  int bad = 0;
  cudaError_t e = cudaMemcpyAsync(&bad, ctx->flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
  if (rc) return rc;
  if (e != cudaSuccess) return fail(ctx, PTYCHO_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  if (bad) return fail(ctx, PTYCHO_ERR_NONFINITE, "%s: frames contain NaN or Inf", what);
  ctx->have_data = true;
  ctx->psi_valid = false;
  return PTYCHO_OK;
}

}  // namespace

extern "C" {

int ptycho_set_data(ptycho_ctx* ctx, const float* intensities, const float* positions, int on_device) {
  if (!ctx) return PTYCHO_ERR_ARG;
  if (!intensities) return fail(ctx, PTYCHO_ERR_ARG, "intensities is NULL");
  if (int r = set_positions_impl(ctx, positions)) return r;
  ctx->have_data = false;
  const int J = ctx->p.J, M = ctx->p.M;
  const size_t MM = (size_t)M * M;
  CK(cudaMemsetAsync(ctx->flag, 0, sizeof(int), ctx->st));
  int rc;
  if (on_device) {
    rc = prepare_amp(ctx, intensities, 0, J);  // read in place
  } else {
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>(J, (128u << 20) / (MM * 4)));  // <= 128 MB
    rc = upload_chunks(ctx, reinterpret_cast<const unsigned char*>(intensities), MM * 4, J, chunk,
                       [&](const void* dev, int j0, int nj) { return prepare_amp(ctx, (const float*)dev, j0, nj); });
  }
  return finish_set_data(ctx, rc, "set_data");
}

int ptycho_set_data_raw(ptycho_ctx* ctx, const void* raw, const ptycho_preprocess* pp, const float* positions,
                        int on_device) {
  if (!ctx) return PTYCHO_ERR_ARG;
  if (!raw || !pp) return fail(ctx, PTYCHO_ERR_ARG, "raw frames or preprocessing parameters are NULL");
  if (pp->raw_h < 1 || pp->raw_w < 1 || pp->dtype < PTYCHO_RAW_U16 || pp->dtype > PTYCHO_RAW_F32 ||
      pp->saturation_bits < 0 || pp->saturation_bits > 24 || pp->rot90 < 0 || pp->rot90 > 3 ||
      !std::isfinite(pp->center_y) || !std::isfinite(pp->center_x) || !std::isfinite(pp->threshold))
    return fail(ctx, PTYCHO_ERR_ARG, "bad preprocessing parameters");
  if (int r = set_positions_impl(ctx, positions)) return r;
  ctx->have_data = false;
  const int J = ctx->p.J, M = ctx->p.M;
  const size_t MM = (size_t)M * M;
  const size_t esz = pp->dtype == PTYCHO_RAW_U16 ? 2 : 4;
  const size_t frame_bytes = (size_t)pp->raw_h * pp->raw_w * esz;
  PreArgs q{};
  q.H = pp->raw_h;
  q.W = pp->raw_w;
  q.cy = (int)std::nearbyint((double)pp->center_y);
  q.cx = (int)std::nearbyint((double)pp->center_x);
  q.M = M;
  q.sat = pp->saturation_bits > 0 ? (float)((1u << pp->saturation_bits) - 1u) : INFINITY;
  q.thr = pp->threshold;
  q.rot = pp->rot90;
  q.bad = ctx->flag;
  // detector-centred intensities of one chunk (<= 128 MB of raw frames and of
  // their preprocessed form), then the amplitude preparation; the same chunk
  // bounds the uploads, so a chunk never exceeds the preprocessing buffer
  const int chunk = (int)std::max<size_t>(1, std::min<size_t>(J, (128u << 20) / std::max(frame_bytes, MM * 4)));
  if (ctx->pre_frames < chunk) {  // none yet, or one for a smaller chunk
    if (ctx->pre) {
      CK(cudaStreamSynchronize(ctx->st));
      dfree(ctx, ctx->pre);
    }
    if (int r = dalloc(ctx, &ctx->pre, (size_t)chunk * MM)) return r;
    ctx->pre_frames = chunk;
  }
  auto process = [&](const void* dev, int j0, int nj) {
    if (nj > ctx->pre_frames) return fail(ctx, PTYCHO_ERR_ARG, "internal: chunk of %d frames exceeds %d", nj, ctx->pre_frames);
    q.raw = dev;
    q.nj = nj;
    q.out = ctx->pre;
    if (int r = launch(ctx, "preprocess", (double)nj * (frame_bytes + MM * 4), [&] {
          const dim3 g((unsigned)M, (unsigned)std::min(nj, 65535));
          if (pp->dtype == PTYCHO_RAW_U16) k_preprocess<unsigned short><<<g, 128, 0, ctx->st>>>(q);
          else if (pp->dtype == PTYCHO_RAW_U32) k_preprocess<unsigned int><<<g, 128, 0, ctx->st>>>(q);
          else k_preprocess<float><<<g, 128, 0, ctx->st>>>(q);
        }))
      return r;
    return prepare_amp(ctx, ctx->pre, j0, nj);
  };
  CK(cudaMemsetAsync(ctx->flag, 0, sizeof(int), ctx->st));
  int rc = 0;
  if (on_device) {
    for (int j0 = 0; j0 < J && !rc; j0 += chunk)
      rc = process(reinterpret_cast<const unsigned char*>(raw) + (size_t)j0 * frame_bytes, j0, std::min(chunk, J - j0));
  } else {
    rc = upload_chunks(ctx, reinterpret_cast<const unsigned char*>(raw), frame_bytes, J, chunk, process);
  }
  return finish_set_data(ctx, rc, "set_data_raw");
}

int ptycho_set_init(ptycho_ctx* ctx, const float* object, const float* probe, int on_device) {
  if (!ctx) return PTYCHO_ERR_ARG;
  const size_t no = object ? (size_t)ctx->p.obj_ny * ctx->p.obj_nx * 2 : 0;
  const size_t np = probe ? (size_t)ctx->p.K * ctx->p.M * ctx->p.M * 2 : 0;
  if (!no && !np) return PTYCHO_OK;
  // the guesses are checked for NaN / Inf on the device before they replace
  // the current state (host inputs go through the staging buffer)
  const float* so = object;
  const float* sp = probe;
  if (!on_device) {
    if (int r = ensure_stage(ctx, (no + np) * 4)) return r;
    if (no) CK(cudaMemcpyAsync(ctx->stage, object, no * 4, cudaMemcpyHostToDevice, ctx->st));
    if (np) CK(cudaMemcpyAsync(ctx->stage + no, probe, np * 4, cudaMemcpyHostToDevice, ctx->st));
    so = ctx->stage;
    sp = ctx->stage + no;
  }
  CK(cudaMemsetAsync(ctx->flag, 0, sizeof(int), ctx->st));
  if (no) k_check_finite<<<592, 256, 0, ctx->st>>>(so, no, ctx->flag);
  if (np) k_check_finite<<<592, 256, 0, ctx->st>>>(sp, np, ctx->flag);
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, ctx->flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (bad) return fail(ctx, PTYCHO_ERR_NONFINITE, "%s guess has NaN/Inf", no && np ? "object or probe" : (no ? "object" : "probe"));
  if (no) CK(cudaMemcpyAsync(ctx->O, so, no * 4, cudaMemcpyDeviceToDevice, ctx->st));
  if (np) CK(cudaMemcpyAsync(ctx->P, sp, np * 4, cudaMemcpyDeviceToDevice, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  ctx->psi_valid = false;
  return PTYCHO_OK;
}

int ptycho_orthogonalize_probe(ptycho_ctx* ctx) {
  if (!ctx) return PTYCHO_ERR_ARG;
  return ortho_step(ctx, ctx->psi_valid);
}

int ptycho_set_likelihood(ptycho_ctx* ctx, int likelihood) {
  if (!ctx) return PTYCHO_ERR_ARG;
  if (likelihood != PTYCHO_LIK_AMPLITUDE && likelihood != PTYCHO_LIK_POISSON)
    return fail(ctx, PTYCHO_ERR_ARG, "likelihood=%d", likelihood);
  ctx->p.likelihood = likelihood;
  return PTYCHO_OK;
}

int ptycho_set_wait_limit(ptycho_ctx* ctx, long long polls) {
  if (!ctx) return PTYCHO_ERR_ARG;
  if (polls < 0) return fail(ctx, PTYCHO_ERR_ARG, "wait limit %lld < 0", polls);
  ctx->wait_limit = (int)std::min<long long>(polls, 1LL << 30);
  return PTYCHO_OK;
}

int ptycho_iterate(ptycho_ctx* ctx, int alg, int n_iter) {
  if (!ctx) return PTYCHO_ERR_ARG;
  if (n_iter < 0) return fail(ctx, PTYCHO_ERR_ARG, "n_iter=%d", n_iter);
  if (!ctx->have_data) return fail(ctx, PTYCHO_ERR_STATE, "iterate before set_data");
  if (alg != PTYCHO_EPIE && alg != PTYCHO_DM && alg != PTYCHO_LSQML)
    return fail(ctx, PTYCHO_ERR_ARG, "unknown algorithm %d", alg);
  if (n_iter == 0) return PTYCHO_OK;
  static const char* names[] = {"epie", "dm", "lsqml"};
  const char* name = names[alg];
  auto run = [&](int n) {
    NvtxRange range(name);
    return alg == PTYCHO_EPIE ? run_epie(ctx, n) : alg == PTYCHO_DM ? run_dm(ctx, n) : run_lsqml(ctx, n);
  };
  const int every = ctx->log_fn ? ctx->log_every : 0;
  if (every <= 0) return run(n_iter);
  // progress reports: n calls of iterate(1) equal one call of n, so the
  // iterations run in pieces that end where a report is due
  for (int done = 0; done < n_iter;) {
    const int n = (int)std::min<long long>(n_iter - done, every - ctx->t % every);
    if (int r = run(n)) return r;
    done += n;
    if (ctx->t % every == 0 || done == n_iter) {
      double E = 0.0;
      if (int r = ptycho_fourier_error(ctx, &E)) return r;
      char b[128];
      snprintf(b, sizeof b, "%s iteration %lld: E = %.9e", name, ctx->t, E);
      ctx->log_fn(ctx->log_user, PTYCHO_LOG_INFO, b);
    }
  }
  return PTYCHO_OK;
}

int ptycho_set_log(ptycho_ctx* ctx, ptycho_log_fn fn, void* user, int error_every) {
  if (!ctx) return PTYCHO_ERR_ARG;
  if (error_every < 0) return fail(ctx, PTYCHO_ERR_ARG, "error_every=%d", error_every);
  ctx->log_fn = fn;
  ctx->log_user = user;
  ctx->log_every = error_every;
  return PTYCHO_OK;
}

int ptycho_get_object(ptycho_ctx* ctx, float* out, int on_device) {
  if (!ctx) return PTYCHO_ERR_ARG;
  if (int r = check_device_flag(ctx)) return r;
  return copy_out(ctx, out, ctx->O, (size_t)ctx->p.obj_ny * ctx->p.obj_nx * 8, on_device);
}

int ptycho_get_probe(ptycho_ctx* ctx, float* out, int on_device) {
  if (!ctx) return PTYCHO_ERR_ARG;
  if (int r = check_device_flag(ctx)) return r;
  return copy_out(ctx, out, ctx->P, (size_t)ctx->p.K * ctx->p.M * ctx->p.M * 8, on_device);
}

int ptycho_get_exit_waves(ptycho_ctx* ctx, float* out, int on_device) {
  if (!ctx) return PTYCHO_ERR_ARG;
  if (!ctx->psi_valid) return fail(ctx, PTYCHO_ERR_STATE, "no DM exit-wave state");
  return copy_out(ctx, out, ctx->X, (size_t)ctx->p.J * ctx->p.K * ctx->p.M * ctx->p.M * 8, on_device);
}

int ptycho_fourier_error(ptycho_ctx* ctx, double* out) {
  if (!ctx) return PTYCHO_ERR_ARG;
  if (!out) return fail(ctx, PTYCHO_ERR_ARG, "out is NULL");
  if (!ctx->have_data) return fail(ctx, PTYCHO_ERR_STATE, "fourier_error before set_data");
  if (int r = launch_fourier(ctx, FM_ERR, nullptr, nullptr, 0, ctx->p.J, "fourier_err")) return r;
  const int n = ctx->p.J * ctx->C;
  if (int r = launch(ctx, "err_final", 0.0, [&] { k_err_final<<<1, 1024, 0, ctx->st>>>(ctx->err_part, n, ctx->err_out); }))
    return r;
  double2 h;
  CK(cudaMemcpyAsync(&h, ctx->err_out, sizeof h, cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (int r = check_device_flag(ctx)) return r;
  const double E = h.y > 0 ? h.x / h.y : 0.0;
  *out = E;
  if (!std::isfinite(E)) return fail(ctx, PTYCHO_ERR_DIVERGED, "Fourier error is not finite");
  return PTYCHO_OK;
}

int ptycho_simulate(ptycho_ctx* ctx, float* out, int on_device) {
  if (!ctx) return PTYCHO_ERR_ARG;
  if (!out) return fail(ctx, PTYCHO_ERR_ARG, "out is NULL");
  if (!ctx->have_pos) return fail(ctx, PTYCHO_ERR_STATE, "simulate before set_positions");
  const size_t n = (size_t)ctx->p.J * ctx->p.M * ctx->p.M;
  float* dst = on_device ? out : nullptr;
  if (!on_device)
    if (int r = dalloc(ctx, &dst, n)) return r;
  int r = launch_fourier(ctx, FM_SIM, nullptr, dst, 0, ctx->p.J, "fourier_sim");
  if (!r && !on_device) r = copy_out(ctx, out, dst, n * 4, 0);
  if (!r) {
    cudaError_t e = cudaStreamSynchronize(ctx->st);
    if (e != cudaSuccess) r = fail(ctx, PTYCHO_ERR_CUDA, "simulate: %s", cudaGetErrorString(e));
  }
  if (!on_device) dfree(ctx, dst);
  return r;
}

int ptycho_fourier_residual(ptycho_ctx* ctx, float* out, int on_device) {
  if (!ctx) return PTYCHO_ERR_ARG;
  if (!out) return fail(ctx, PTYCHO_ERR_ARG, "out is NULL");
  if (!ctx->have_data) return fail(ctx, PTYCHO_ERR_STATE, "residual before set_data");
  const size_t n = (size_t)ctx->p.J * ctx->p.K * ctx->p.M * ctx->p.M;
  float2* dst = on_device ? (float2*)out : nullptr;
  if (!on_device)
    if (int r = dalloc(ctx, &dst, n)) return r;
  int r = launch_chi(ctx, dst);
  if (!r && !on_device) r = copy_out(ctx, out, dst, n * 8, 0);
  if (!r) {
    cudaError_t e = cudaStreamSynchronize(ctx->st);
    if (e != cudaSuccess) r = fail(ctx, PTYCHO_ERR_CUDA, "residual: %s", cudaGetErrorString(e));
  }
  if (!on_device) dfree(ctx, dst);
  return r;
}

int ptycho_refine_positions(ptycho_ctx* ctx, double step, double max_shift) {
  if (!ctx) return PTYCHO_ERR_ARG;
  if (!ctx->S) return fail(ctx, PTYCHO_ERR_UNSUPPORTED, "position refinement needs sub-pixel positions (subpixel > 0)");
  if (!ctx->have_data) return fail(ctx, PTYCHO_ERR_STATE, "refine_positions before set_data");
  if (!std::isfinite(step) || !(max_shift >= 0.0) || !std::isfinite(max_shift))
    return fail(ctx, PTYCHO_ERR_ARG, "step=%g max_shift=%g", step, max_shift);
  if (int r = ensure_work_buffers(ctx)) return r;
  ctx->psi_valid = false;  // the residual pass overwrites the exit-wave state
  if (int r = launch_chi(ctx, ctx->X)) return r;
  PosCorrArgs a{};
  a.O = ctx->O;
  a.ny = ctx->p.obj_ny;
  a.nx = ctx->p.obj_nx;
  a.P = ctx->Pt;
  a.pbin = ctx->pbin;
  a.X = ctx->X;
  a.pos = ctx->pos;
  a.M = ctx->p.M;
  a.out = ctx->pos_corr;
  const int J = ctx->p.J;
  const double xb = 8.0 * J * ctx->p.K * (double)ctx->p.M * ctx->p.M;
  int r = launch(ctx, "pos_corr", xb, [&] {
    switch (ctx->p.K) {
      case 1: k_pos_corr<1><<<J, STEP_NT, 0, ctx->st>>>(a); break;
      case 2: k_pos_corr<2><<<J, STEP_NT, 0, ctx->st>>>(a); break;
      default: k_pos_corr<3><<<J, STEP_NT, 0, ctx->st>>>(a); break;
    }
  });
  if (r) return r;
  std::vector<float2> s(J);
  CK(cudaMemcpyAsync(s.data(), ctx->pos_corr, J * sizeof(float2), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (int rc = check_device_flag(ctx)) return rc;
  std::vector<float> next(ctx->pos_f);
  for (int j = 0; j < J; ++j) {
    const double sy = std::min(std::max((double)s[j].x, -max_shift), max_shift);
    const double sx = std::min(std::max((double)s[j].y, -max_shift), max_shift);
    if (!std::isfinite(sy) || !std::isfinite(sx))
      return fail(ctx, PTYCHO_ERR_NONFINITE, "position correction of %d is not finite", j);
    next[2 * j] = (float)((double)next[2 * j] + step * sy);
    next[2 * j + 1] = (float)((double)next[2 * j + 1] + step * sx);
  }
  return set_positions_impl(ctx, next.data());  // checks bounds; unchanged on error
}

int ptycho_get_positions(ptycho_ctx* ctx, float* out) {
  if (!ctx) return PTYCHO_ERR_ARG;
  if (!out) return fail(ctx, PTYCHO_ERR_ARG, "out is NULL");
  if (!ctx->have_pos) return fail(ctx, PTYCHO_ERR_STATE, "no positions set");
  std::memcpy(out, ctx->pos_f.data(), ctx->pos_f.size() * sizeof(float));
  return PTYCHO_OK;
}

long long ptycho_iteration(const ptycho_ctx* ctx) { return ctx ? ctx->t : -1; }

int ptycho_set_iteration(ptycho_ctx* ctx, long long t) {
  if (!ctx) return PTYCHO_ERR_ARG;
  if (t < 0) return fail(ctx, PTYCHO_ERR_ARG, "iteration index %lld", t);
  ctx->t = t;
  return PTYCHO_OK;
}

int ptycho_set_exit_waves(ptycho_ctx* ctx, const float* psi, int on_device) {
  if (!ctx) return PTYCHO_ERR_ARG;
  if (!psi) return fail(ctx, PTYCHO_ERR_ARG, "psi is NULL");
  if (int r = ensure_work_buffers(ctx)) return r;
  const size_t n = (size_t)ctx->p.J * ctx->p.K * ctx->p.M * ctx->p.M * 2;  // floats
  // checked for NaN / Inf before it replaces the state (host data through the
  // staging buffer)
  const float* src = psi;
  if (!on_device) {
    if (int r = ensure_stage(ctx, n * 4)) return r;
    CK(cudaMemcpyAsync(ctx->stage, psi, n * 4, cudaMemcpyHostToDevice, ctx->st));
    src = ctx->stage;
  }
  CK(cudaMemsetAsync(ctx->flag, 0, sizeof(int), ctx->st));
  k_check_finite<<<1184, 256, 0, ctx->st>>>(src, n, ctx->flag);
  int bad = 0;
  CK(cudaMemcpyAsync(&bad, ctx->flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  if (bad) return fail(ctx, PTYCHO_ERR_NONFINITE, "exit waves contain NaN/Inf");
  CK(cudaMemcpyAsync(ctx->X, src, n * 4, cudaMemcpyDeviceToDevice, ctx->st));
  CK(cudaStreamSynchronize(ctx->st));
  ctx->psi_valid = true;
  return PTYCHO_OK;
}
long long ptycho_launch_count(const ptycho_ctx* ctx) { return ctx ? ctx->launches : -1; }
long long ptycho_memory_used(const ptycho_ctx* ctx) { return ctx ? (long long)ctx->mem_used : -1; }
int ptycho_cluster_size(const ptycho_ctx* ctx) { return ctx ? ctx->C : 0; }
int ptycho_epie_cluster_size(const ptycho_ctx* ctx) {
  if (!ctx) return 0;
  if (ctx->S) return ctx->fks_one ? ctx->fks_one->C : ctx->C;
  return ctx->eks && ctx->epie_ok ? ctx->eks->C : 0;
}

int ptycho_set_profiling(ptycho_ctx* ctx, int enabled) {
  if (!ctx) return PTYCHO_ERR_ARG;
  if (int r = collect_profile(ctx)) return r;
  ctx->prof = enabled != 0;
  for (auto& s : ctx->stats) s = ptycho_kernel_stat{};
  return PTYCHO_OK;
}

int ptycho_get_profile(ptycho_ctx* ctx, ptycho_kernel_stat* out, int max, int* n) {
  if (!ctx) return PTYCHO_ERR_ARG;
  if (int r = collect_profile(ctx)) return r;
  const int nf = (int)ctx->stats.size();
  for (int i = 0; i < nf && i < max && out; ++i) {
    out[i] = ctx->stats[i];
    out[i].name = ctx->fam_names[i].c_str();
  }
  if (n) *n = nf;
  return PTYCHO_OK;
}

const char* ptycho_last_error(const ptycho_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

void ptycho_destroy(ptycho_ctx* ctx) {
  if (!ctx) return;
  if (ctx->st) cudaStreamSynchronize(ctx->st);
  else cudaDeviceSynchronize();
  if (ctx->st_side) {  // its work is joined into ctx->st, which is idle now
    cudaStreamSynchronize(ctx->st_side);
    cudaStreamDestroy(ctx->st_side);
  }
  if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
  if (ctx->ev_join) cudaEventDestroy(ctx->ev_join);
  void* bufs[] = {ctx->tw2, ctx->err_flag, ctx->O,        ctx->P,         ctx->X,        ctx->dO,       ctx->dP,        ctx->tw,
                  ctx->pos,      ctx->amp,       ctx->amp_scale, ctx->denO,    ctx->tile_max,  ctx->denO_max,
                  ctx->tile_ptr, ctx->tile_list, ctx->ppart,    ctx->ppart_den, ctx->pnum,     ctx->pden,
                  ctx->pblk_max, ctx->alphaO,    ctx->alphaP,   ctx->err_part, ctx->err_out,   ctx->order,
                  ctx->flag,     ctx->gram,      ctx->modeV,    ctx->pbin,     ctx->Pt,        ctx->dPt,
                  ctx->pbins,    ctx->stmp,      ctx->porder,   ctx->goff,     ctx->bgrp,
                  ctx->pbins_den, ctx->cg_r,     ctx->cg_p,     ctx->cg_q,     ctx->cg_part,
                  ctx->pos_corr, ctx->objacc, ctx->ep_mx, ctx->dftm};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (ctx->stage) cudaFree(ctx->stage);
  if (ctx->pre) cudaFree(ctx->pre);
  if (ctx->st_copy) {
    cudaStreamSynchronize(ctx->st_copy);
    cudaStreamDestroy(ctx->st_copy);
  }
  for (int h = 0; h < 2; ++h) {
    if (ctx->ev_copied[h]) cudaEventDestroy(ctx->ev_copied[h]);
    if (ctx->ev_used[h]) cudaEventDestroy(ctx->ev_used[h]);
  }
  for (auto& r : ctx->pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : ctx->ev_pool) cudaEventDestroy(e);
  delete ctx;
}

}  // extern "C"

#include "batch.cuh"
#include "net_api.cuh"

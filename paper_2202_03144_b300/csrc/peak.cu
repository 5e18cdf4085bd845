// FP32 fused multiply-add throughput of the current device, measured.
//
// The roofline of the instruction-bound Fourier passes is quoted against the
// FP32 rate this kernel reaches, not against a figure derived from unit
// counts: every thread runs NCH independent FMA chains (enough independent
// work per warp to cover the FMA latency), the grid fills every SM several
// times over, and the kernel is timed with CUDA events on the caller's
// stream.  Two flops per FMA.
#include <cuda_runtime.h>

#include "../../include/ptycho.h"

namespace {

constexpr int PEAK_NT = 256;
constexpr int PEAK_NCH = 8;      // independent chains per thread
constexpr int PEAK_UNROLL = 64;  // FMAs per chain per loop trip

__global__ void __launch_bounds__(PEAK_NT) k_fma_peak(float* out, int trips, float a, float b) {
  float x[PEAK_NCH];
#pragma unroll
  for (int c = 0; c < PEAK_NCH; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
  for (int t = 0; t < trips; ++t) {
#pragma unroll
    for (int u = 0; u < PEAK_UNROLL; ++u)
#pragma unroll
      for (int c = 0; c < PEAK_NCH; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < PEAK_NCH; ++c) s += x[c];
  // a contraction |a| < 1 keeps every value finite; the store keeps the work
  if (s == 12345.678f) out[blockIdx.x * PEAK_NT + threadIdx.x] = s;
}

}  // namespace

extern "C" int ptycho_fp32_fma_peak(double* tflops, double* ms, int* sm_count, void* stream) {
  if (!tflops) return PTYCHO_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PTYCHO_ERR_CUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PTYCHO_ERR_CUDA;
  const int blocks = sms * 8;     // 8 x 256 threads resident per SM: every scheduler busy
  const int trips = 2048;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return PTYCHO_ERR_CUDA;
  float best = 0.f;
  bool ok = true;
  for (int rep = 0; rep < 4 && ok; ++rep) {  // the first run warms clocks and caches
    cudaEventRecord(e0, st);
    k_fma_peak<<<blocks, PEAK_NT, 0, st>>>(nullptr, trips, 0.999f, 1e-4f);
    cudaEventRecord(e1, st);
    ok = cudaEventSynchronize(e1) == cudaSuccess && cudaGetLastError() == cudaSuccess;
    float t = 0.f;
    if (ok && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess && rep > 0 && (best == 0.f || t < best)) best = t;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!ok || best <= 0.f) return PTYCHO_ERR_CUDA;
  const double flops = 2.0 * PEAK_NCH * PEAK_UNROLL * (double)trips * blocks * PEAK_NT;
  *tflops = flops / (best * 1e-3) / 1e12;
  if (ms) *ms = best;
  if (sm_count) *sm_count = sms;
  return PTYCHO_OK;
}

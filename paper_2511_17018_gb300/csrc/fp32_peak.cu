// FP32 throughput microbenchmark: the measured peak the fit's throughput is
// reported against.  Every thread runs kChains independent FMA chains (enough
// independent work per warp to cover the FMA latency), the grid fills every
// SM with 2,048 threads, and the time of one launch is taken with CUDA events
// on the caller's stream.  Mode 0 issues scalar fma.rn.f32, mode 1 the paired
// fma.rn.f32x2 (two lanes' worth of FP32 work per instruction).
#include <cuda_runtime.h>

#include <cstdint>

#include "tpcfit.h"

namespace tpcfit {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 32;
constexpr int kThreads = 512;
constexpr int kBlocksPerSm = 4;

// Where a chain's result would go; the kernels never take that branch (the
// chains stay positive), it only keeps the compiler from removing them.
__device__ float g_sink[kThreads];

__global__ void __launch_bounds__(kThreads) ffma_chains(int64_t iters, float b, float c) {
  float a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
#pragma unroll 1
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) a[k] = fmaf(a[k], b, c);
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s == -1.0f) g_sink[threadIdx.x] = s;
}

__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

__global__ void __launch_bounds__(kThreads) ffma2_chains(int64_t iters, float b, float c) {
  unsigned long long a[kChains / 2];
  const unsigned long long bb = ((unsigned long long)__float_as_uint(b) << 32) | __float_as_uint(b);
  const unsigned long long cc = ((unsigned long long)__float_as_uint(c) << 32) | __float_as_uint(c);
#pragma unroll
  for (int k = 0; k < kChains / 2; ++k) {
    const unsigned lo = __float_as_uint((float)(threadIdx.x + 2 * k) * 1e-3f);
    const unsigned hi = __float_as_uint((float)(threadIdx.x + 2 * k + 1) * 1e-3f);
    a[k] = ((unsigned long long)hi << 32) | lo;
  }
#pragma unroll 1
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kChains / 2; ++k) a[k] = fma2(a[k], bb, cc);
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains / 2; ++k)
    s += __uint_as_float((unsigned)(a[k] & 0xffffffffull)) + __uint_as_float((unsigned)(a[k] >> 32));
  if (s == -1.0f) g_sink[threadIdx.x] = s;
}

}  // namespace
}  // namespace tpcfit

extern "C" tpcfit_status tpcfit_fp32_peak(int mode, int64_t iterations, void* stream, double* flop_out,
                                          double* ms_out) {
  using namespace tpcfit;
  if ((mode != 0 && mode != 1) || iterations < 1 || !flop_out || !ms_out) return TPCFIT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return TPCFIT_ECUDA;
  const int blocks = sms * kBlocksPerSm;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  if (e == cudaSuccess) {
    // warm-up launch, then the timed one
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
      const int64_t it = rep == 0 ? (iterations < 64 ? iterations : 64) : iterations;
      if (rep == 1) e = cudaEventRecord(t0, s);
      if (e != cudaSuccess) break;
      if (mode == 0) ffma_chains<<<blocks, kThreads, 0, s>>>(it, 0.9999f, 1e-4f);
      else ffma2_chains<<<blocks, kThreads, 0, s>>>(it, 0.9999f, 1e-4f);
      e = cudaGetLastError();
    }
  }
  if (e == cudaSuccess) e = cudaEventRecord(t1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(t1);
  float ms = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (e != cudaSuccess) return TPCFIT_ECUDA;
  *flop_out = 2.0 * (double)kChains * (double)kUnroll * (double)iterations * (double)blocks * (double)kThreads;
  *ms_out = (double)ms;
  return TPCFIT_OK;
}

// Track ordering by length: a counting sort over the number of clusters per
// track, longest first, so that the 32 tracks of a warp have equal lengths and
// its lanes finish together.  Positions within one length are assigned with
// atomics; the fit writes every output at the track's own index, so the
// results do not depend on that order.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "device_util.cuh"

namespace tpcfit {
namespace {

constexpr int kBins = 256;
constexpr int kThreads = 256;
constexpr int kItems = 4;

__device__ __forceinline__ int length_bin(const int32_t* off, int64_t i) {
  int len = off[i + 1] - off[i];
  return len < 0 ? 0 : (len > kBins - 1 ? kBins - 1 : len);
}

__global__ void __launch_bounds__(kThreads) length_hist(const int32_t* off, int32_t n, int32_t* hist) {
  __shared__ int sh[kBins];
  for (int i = threadIdx.x; i < kBins; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kThreads * kItems;
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const int64_t i = base + (int64_t)it * kThreads + threadIdx.x;
    if (i < n) atomicAdd(&sh[length_bin(off, i)], 1);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kBins; b += blockDim.x)
    if (sh[b]) atomicAdd(&hist[b], sh[b]);
}

__global__ void __launch_bounds__(kThreads) length_scatter(const int32_t* off, int32_t n, const int32_t* hist,
                                                           int32_t* cursor, int32_t* perm) {
  __shared__ int start[kBins];
  __shared__ int local[kBins];
  __shared__ int base[kBins];
  {
    // start[b] = number of tracks longer than b (longest first)
    const int b = threadIdx.x;
    int acc = 0;
    for (int L = kBins - 1; L > b; --L) acc += hist[L];
    start[b] = acc;
    local[b] = 0;
  }
  __syncthreads();
  const int64_t first = (int64_t)blockIdx.x * kThreads * kItems;
  int bin[kItems], rank[kItems];
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const int64_t i = first + (int64_t)it * kThreads + threadIdx.x;
    bin[it] = -1;
    if (i < n) {
      bin[it] = length_bin(off, i);
      rank[it] = atomicAdd(&local[bin[it]], 1);
    }
  }
  __syncthreads();
  {
    const int b = threadIdx.x;
    base[b] = local[b] ? atomicAdd(&cursor[b], local[b]) : 0;
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const int64_t i = first + (int64_t)it * kThreads + threadIdx.x;
    if (bin[it] >= 0) perm[start[bin[it]] + base[bin[it]] + rank[it]] = (int32_t)i;
  }
}

// Batched frames: key = frame * 256 + (255 - length) orders by frame, then by
// decreasing length.  Histogram with global atomics, exclusive scan, scatter.
__device__ __forceinline__ int frame_key(const int32_t* off, const int64_t* fb, int n_frames, int64_t i) {
  int f = frame_of(fb, n_frames, i);
  if (f < 0) f = n_frames - 1;  // out-of-table tracks are rejected by the fit; keep them in range here
  return f * kBins + (kBins - 1 - length_bin(off, i));
}

__global__ void frame_hist(const int32_t* off, int32_t n, const int64_t* fb, int n_frames, int32_t* hist) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&hist[frame_key(off, fb, n_frames, i)], 1);
}

__global__ void frame_scatter(const int32_t* off, int32_t n, const int64_t* fb, int n_frames, const int32_t* start,
                              int32_t* cursor, int32_t* perm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int k = frame_key(off, fb, n_frames, i);
  perm[start[k] + atomicAdd(&cursor[k], 1)] = (int32_t)i;
}

}  // namespace

int64_t frame_order_scratch_ints(int32_t n_frames) {
  const int64_t bins = (int64_t)n_frames * kBins;
  return 2 * bins + scan_tmp_ints(bins);
}

cudaError_t launch_frame_length_order(const int32_t* off, int32_t n_tracks, const int64_t* frame_base,
                                      int32_t n_frames, int32_t* perm, int32_t* scratch, cudaStream_t s) {
  if (n_tracks <= 0) return cudaSuccess;
  const int64_t bins = (int64_t)n_frames * kBins;
  int32_t* start = scratch;
  int32_t* cursor = scratch + bins;
  int32_t* tmp = scratch + 2 * bins;
  cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(int32_t) * 2 * bins, s);
  if (e != cudaSuccess) return e;
  const int64_t blocks = ((int64_t)n_tracks + 255) / 256;
  frame_hist<<<(unsigned)blocks, 256, 0, s>>>(off, n_tracks, frame_base, n_frames, start);
  e = launch_scan_exclusive(start, (int)bins, tmp, s);
  if (e != cudaSuccess) return e;
  frame_scatter<<<(unsigned)blocks, 256, 0, s>>>(off, n_tracks, frame_base, n_frames, start, cursor, perm);
  return cudaGetLastError();
}

cudaError_t launch_length_order(const int32_t* off, int32_t n_tracks, int32_t* perm, int32_t* scratch,
                                cudaStream_t s) {
  if (n_tracks <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(int32_t) * 2 * kBins, s);
  if (e != cudaSuccess) return e;
  const int64_t blocks = ((int64_t)n_tracks + kThreads * kItems - 1) / (kThreads * kItems);
  length_hist<<<(unsigned)blocks, kThreads, 0, s>>>(off, n_tracks, scratch);
  length_scatter<<<(unsigned)blocks, kThreads, 0, s>>>(off, n_tracks, scratch, scratch + kBins, perm);
  return cudaGetLastError();
}

}  // namespace tpcfit

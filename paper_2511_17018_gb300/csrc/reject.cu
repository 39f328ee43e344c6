// Outlier rejection after the smoother: every cluster whose leave-one-out
// chi2 exceeds a cut is dropped from its track, the others are copied in
// their order.  One warp per track; the kept clusters of 32 consecutive
// clusters are placed with a ballot and a population count, so the output
// order is the input order (the cluster-to-track relation the deterministic
// mode keeps, Sec. 2) and the results do not depend on scheduling.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace tpcfit {
namespace {

constexpr int kWarpsPerBlock = 8;

// A cluster is kept unless its chi2 is above the cut; a NaN chi2 (no
// leave-one-out estimate) keeps it.
__device__ __forceinline__ bool keep_cluster(const float* chi2, int64_t c, float cut) { return !(chi2[c] > cut); }

// Cluster range of track t, empty if the offsets are out of order or outside
// the cluster arrays.
__device__ __forceinline__ void track_range(const int32_t* off, int32_t t, int64_t n_hits, int32_t& b, int32_t& e) {
  b = off[t];
  e = off[t + 1];
  if (b < 0 || e < b || (int64_t)e > n_hits) b = e = 0;
}

// kept[t] = number of clusters track t keeps; kept[n_tracks] = 0 (the scan
// turns the array into the new offsets).
__global__ void __launch_bounds__(kWarpsPerBlock * 32) reject_count(const int32_t* off, int32_t n_tracks,
                                                                      int64_t n_hits, const float* chi2, float cut,
                                                                      int32_t* kept) {
  const int64_t t = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (t == 0 && lane == 0) kept[n_tracks] = 0;
  if (t >= n_tracks) return;
  int32_t b, e;
  track_range(off, (int32_t)t, n_hits, b, e);
  int n = 0;
  for (int32_t base = b; base < e; base += 32) {
    const int32_t c = base + lane;
    const bool k = c < e && keep_cluster(chi2, c, cut);
    n += __popc(__ballot_sync(0xffffffffu, k));
  }
  if (lane == 0) kept[t] = n;
}

// Copy the kept clusters of track t to start new_off[t], in order; nothing
// is written at or beyond n_hits (the outputs' length).
__global__ void __launch_bounds__(kWarpsPerBlock * 32) reject_compact(
    const int32_t* off, int32_t n_tracks, int64_t n_hits, const float* chi2, float cut, const float* y,
    const float* z, const uint16_t* rowsec, const int32_t* new_off, float* y_out, float* z_out,
    uint16_t* rowsec_out) {
  const int64_t t = (int64_t)blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= n_tracks) return;
  int32_t b, e;
  track_range(off, (int32_t)t, n_hits, b, e);
  int32_t pos = new_off[t];
  const unsigned below = (1u << lane) - 1u;
  for (int32_t base = b; base < e; base += 32) {
    const int32_t c = base + lane;
    const bool k = c < e && keep_cluster(chi2, c, cut);
    const unsigned m = __ballot_sync(0xffffffffu, k);
    const int32_t o = pos + __popc(m & below);
    if (k && o >= 0 && (int64_t)o < n_hits) {  // overlapping ranges must not write outside the outputs
      y_out[o] = y[c];
      z_out[o] = z[c];
      rowsec_out[o] = rowsec[c];
    }
    pos += __popc(m);
  }
}

}  // namespace

int64_t reject_scratch_ints(int32_t n_tracks) { return scan_tmp_ints((int64_t)n_tracks + 1); }

cudaError_t launch_reject(const int32_t* off, int32_t n_tracks, const float* y, const float* z, const uint16_t* rowsec,
                          int64_t n_hits, const float* chi2, float cut, float* y_out, float* z_out,
                          uint16_t* rowsec_out, int32_t* off_out, int32_t* scratch, cudaStream_t s) {
  if (n_tracks <= 0) return cudaMemsetAsync(off_out, 0, sizeof(int32_t), s);
  const unsigned blocks = (unsigned)(((int64_t)n_tracks + kWarpsPerBlock - 1) / kWarpsPerBlock);
  reject_count<<<blocks, kWarpsPerBlock * 32, 0, s>>>(off, n_tracks, n_hits, chi2, cut, off_out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_scan_exclusive(off_out, n_tracks + 1, scratch, s);
  if (e != cudaSuccess) return e;
  reject_compact<<<blocks, kWarpsPerBlock * 32, 0, s>>>(off, n_tracks, n_hits, chi2, cut, y, z, rowsec, off_out, y_out,
                                                        z_out, rowsec_out);
  return cudaGetLastError();
}

}  // namespace tpcfit

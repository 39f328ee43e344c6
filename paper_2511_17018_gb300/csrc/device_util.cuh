// Small device helpers shared by the kernel modules.
#pragma once

#ifndef __CUDACC_RTC__
#include <cuda_runtime.h>
#include <stdint.h>
#endif

namespace tpcfit {

// Frame of track `trk`: f with base[f] <= trk < base[f + 1] (base[0] = 0,
// base[n_frames] = total tracks); -1 if trk lies outside the table.
__device__ __forceinline__ int frame_of(const int64_t* base, int n_frames, int64_t trk) {
  if (trk < __ldg(base) || trk >= __ldg(base + n_frames)) return -1;
  int lo = 0, hi = n_frames;  // invariant: base[lo] <= trk < base[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(base + mid) <= trk) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait until *flag != 0 (acquire), for at most timeout_ns of device time and at
// most 2^23 polls.  Returns false if the wait ran out.
__device__ __forceinline__ bool wait_flag(const int32_t* flag, int64_t timeout_ns) {
  const uint64_t t0 = global_ns();
#pragma unroll 1
  for (int it = 0; it < (1 << 23); ++it) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(flag) : "memory");
    if (v != 0) return true;
    if ((int64_t)(global_ns() - t0) > timeout_ns) return false;
    __nanosleep(256);
  }
  return false;
}

}  // namespace tpcfit

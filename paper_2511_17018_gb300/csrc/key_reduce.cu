// Deterministic reduction of per-cluster gradients into per-(sector, row)
// alignment gradients: the "additional sorting kernels" and fixed-order
// processing of the deterministic mode (Sec. 2).
//
// 1. key_sort: a stable least-significant-digit radix sort (two passes of 7
//    bits over key = sector * 152 + row) of the cluster indices.  Stability
//    comes from ranking the elements of a block in element order (round, warp,
//    lane) with warp match masks and per-warp counts combined in warp order.
// 2. key_reduce: one warp per key sums its clusters' gradients in sorted order:
//    lane l takes every 32nd element starting at l, then a fixed shuffle tree.
// The order of every floating-point addition is a function of the input only.
//
// The default reduction is order-independent instead (key_fixed_*): every
// per-cluster gradient is rounded once to a 64-bit fixed-point integer whose
// unit is a power of two, 2^-S, fixed by the largest finite |gradient| of the
// call and by the number of clusters, so that no sum can overflow; integer
// addition is associative, so the sums do not depend on the order in which
// blocks, warps and atomics add them, and each key's result (the integer sum
// times 2^-S, rounded once to FP32) is the same bits in every run.  The
// rounding to 2^-S is at most 2^-(63 - ceil(log2(n_hits + 1))) of the largest
// |gradient| per cluster, far below the FP32 rounding of a sum.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace tpcfit {
namespace {

constexpr int kKeys = kNSectors * kMaxRows;  // 5472
constexpr int kKeyInvalid = kKeys;            // clusters with an invalid row/sector
constexpr int kDigits = 128;                  // 7 bits per pass
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 8;                     // elements per thread per block
constexpr int kTile = kThreads * kItems;      // 2048

__device__ __forceinline__ int cluster_key(const uint16_t* rowsec, int h, int n_rows) {
  const int rs = (int)__ldg(rowsec + h);
  const int row = rs >> 6, sec = rs & 63;
  return (row < n_rows && sec < kNSectors) ? sec * kMaxRows + row : kKeyInvalid;
}

__device__ __forceinline__ int digit_of(int key, int pass) { return pass == 0 ? (key & 127) : (key >> 7); }

// counts[d * nblocks + b] = number of elements of block b with digit d
__global__ void __launch_bounds__(kThreads) radix_hist(const uint16_t* rowsec, int n, int n_rows, const int* in,
                                                       int pass, int* counts, int nblocks) {
  __shared__ int sh[kDigits];
  for (int i = threadIdx.x; i < kDigits; i += kThreads) sh[i] = 0;
  __syncthreads();
  const int base = blockIdx.x * kTile;
#pragma unroll
  for (int it = 0; it < kItems; ++it) {
    const int j = base + it * kThreads + threadIdx.x;
    if (j < n) {
      const int h = in ? in[j] : j;
      atomicAdd(&sh[digit_of(cluster_key(rowsec, h, n_rows), pass)], 1);
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kDigits; d += kThreads) counts[d * nblocks + blockIdx.x] = sh[d];
}

// Exclusive scan in three phases: per-tile scans (2048 ints per block, in
// shared memory), one block scanning the tile totals, then the tile offsets.
constexpr int kScanTile = 2048;

__device__ __forceinline__ int block_exclusive_scan_2048(int* sh, int tid) {
  // sh[0..2047], 1024 threads, two elements each; returns the tile total
  const int a = sh[2 * tid], b = sh[2 * tid + 1];
  __shared__ int part[1024];
  part[tid] = a + b;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int t = tid >= off ? part[tid - off] : 0;
    __syncthreads();
    part[tid] += t;
    __syncthreads();
  }
  const int excl = tid ? part[tid - 1] : 0;
  const int total = part[1023];
  sh[2 * tid] = excl;
  sh[2 * tid + 1] = excl + a;
  __syncthreads();
  return total;
}

__global__ void __launch_bounds__(1024) scan_tiles(int* v, int n, int* tile_tot) {
  __shared__ int sh[kScanTile];
  const int base = blockIdx.x * kScanTile;
  for (int i = threadIdx.x; i < kScanTile; i += 1024) sh[i] = base + i < n ? v[base + i] : 0;
  __syncthreads();
  const int total = block_exclusive_scan_2048(sh, threadIdx.x);
  for (int i = threadIdx.x; i < kScanTile; i += 1024)
    if (base + i < n) v[base + i] = sh[i];
  if (threadIdx.x == 0) tile_tot[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) scan_totals(int* tot, int n_tiles) {
  // sequential over chunks of 2048 tiles, carrying the running sum
  __shared__ int sh[kScanTile];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n_tiles; base += kScanTile) {
    for (int i = threadIdx.x; i < kScanTile; i += 1024) sh[i] = base + i < n_tiles ? tot[base + i] : 0;
    __syncthreads();
    const int total = block_exclusive_scan_2048(sh, threadIdx.x);
    const int c = carry;
    for (int i = threadIdx.x; i < kScanTile; i += 1024)
      if (base + i < n_tiles) tot[base + i] = sh[i] + c;
    __syncthreads();
    if (threadIdx.x == 0) carry = c + total;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(1024) scan_add(int* v, int n, const int* tile_off) {
  const int base = blockIdx.x * kScanTile;
  const int add = tile_off[blockIdx.x];
  for (int i = threadIdx.x; i < kScanTile; i += 1024)
    if (base + i < n) v[base + i] += add;
}

__global__ void __launch_bounds__(kThreads) radix_scatter(const uint16_t* rowsec, int n, int n_rows, const int* in,
                                                          int* out, int pass, const int* offsets, int nblocks) {
  __shared__ int run[kDigits];               // running count per digit within the block
  __shared__ int wcount[kWarps][kDigits];    // per-warp counts of the current round
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kDigits; i += kThreads) run[i] = 0;
  const int base = blockIdx.x * kTile;
#pragma unroll 1
  for (int it = 0; it < kItems; ++it) {
    for (int i = threadIdx.x; i < kWarps * kDigits; i += kThreads) (&wcount[0][0])[i] = 0;
    __syncthreads();
    const int j = base + it * kThreads + threadIdx.x;
    const bool valid = j < n;
    const int h = valid ? (in ? in[j] : j) : 0;
    const int d = valid ? digit_of(cluster_key(rowsec, h, n_rows), pass) : kDigits;  // kDigits: no digit
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wcount[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      int before = run[d];
      for (int w = 0; w < warp; ++w) before += wcount[w][d];
      out[offsets[d * nblocks + blockIdx.x] + before + rank] = h;
    }
    __syncthreads();
    for (int dd = threadIdx.x; dd < kDigits; dd += kThreads) {
      int add = 0;
      for (int w = 0; w < kWarps; ++w) add += wcount[w][dd];
      run[dd] += add;
    }
    __syncthreads();
  }
}

// key_start[k] = first sorted position with key >= k (k = 0..kKeys)
__global__ void key_bounds(const uint16_t* rowsec, const int* sorted, int n, int n_rows, int* key_start) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j > n) return;
  const int kcur = j < n ? cluster_key(rowsec, sorted[j], n_rows) : kKeys + 1;
  const int kprev = j > 0 ? cluster_key(rowsec, sorted[j - 1], n_rows) : -1;
  for (int k = kprev + 1; k <= kcur && k <= kKeys; ++k) key_start[k] = j;
}

__global__ void __launch_bounds__(256) key_sum(const float* gm, const int* sorted, const int* key_start,
                                               float* grad_align) {
  const int key = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (key >= kKeys) return;
  const int b = key_start[key], e = key_start[key + 1];
  float sy = 0.0f, sz = 0.0f;
  for (int j = b + lane; j < e; j += 32) {
    const float2 g = reinterpret_cast<const float2*>(gm)[sorted[j]];
    sy = sy + g.x;
    sz = sz + g.y;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    sy = sy + __shfl_down_sync(0xffffffffu, sy, off);
    sz = sz + __shfl_down_sync(0xffffffffu, sz, off);
  }
  if (lane == 0) {
    grad_align[key * 2] = -sy;
    grad_align[key * 2 + 1] = -sz;
  }
}

}  // namespace

size_t key_sort_scratch_bytes(int64_t n_hits) {
  const int64_t nblocks = (n_hits + kTile - 1) / kTile;
  const int64_t ncount = kDigits * nblocks;
  return sizeof(int) * (size_t)(2 * n_hits + ncount + (ncount + kScanTile - 1) / kScanTile + kKeys + 2);
}

// Sort cluster indices by key (stable) into `sorted` and fill key_start.
cudaError_t launch_key_sort(const uint16_t* rowsec, int64_t n_hits, int n_rows, void* scratch, int** sorted_out,
                            int** key_start_out, cudaStream_t s) {
  const int n = (int)n_hits;
  const int nblocks = (n + kTile - 1) / kTile;
  int* a = static_cast<int*>(scratch);
  int* b = a + n_hits;
  int* counts = b + n_hits;
  const int ncount = kDigits * nblocks;
  const int n_tiles = (ncount + kScanTile - 1) / kScanTile;
  int* tile_tot = counts + ncount;
  int* key_start = tile_tot + n_tiles;
  *sorted_out = b;
  *key_start_out = key_start;
  if (n == 0) return cudaMemsetAsync(key_start, 0, sizeof(int) * (kKeys + 2), s);
  const int* in = nullptr;
  int* outs[2] = {a, b};
  for (int pass = 0; pass < 2; ++pass) {
    radix_hist<<<nblocks, kThreads, 0, s>>>(rowsec, n, n_rows, in, pass, counts, nblocks);
    scan_tiles<<<n_tiles, 1024, 0, s>>>(counts, ncount, tile_tot);
    scan_totals<<<1, 1024, 0, s>>>(tile_tot, n_tiles);
    scan_add<<<n_tiles, 1024, 0, s>>>(counts, ncount, tile_tot);
    radix_scatter<<<nblocks, kThreads, 0, s>>>(rowsec, n, n_rows, in, outs[pass], pass, counts, nblocks);
    in = outs[pass];
  }
  key_bounds<<<(n + 1 + 255) / 256, 256, 0, s>>>(rowsec, b, n, n_rows, key_start);
  return cudaGetLastError();
}

int64_t scan_tmp_ints(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

cudaError_t launch_scan_exclusive(int* v, int n, int* tmp, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int n_tiles = (n + kScanTile - 1) / kScanTile;
  scan_tiles<<<n_tiles, 1024, 0, s>>>(v, n, tmp);
  scan_totals<<<1, 1024, 0, s>>>(tmp, n_tiles);
  scan_add<<<n_tiles, 1024, 0, s>>>(v, n, tmp);
  return cudaGetLastError();
}

namespace {

// Largest finite |g| over the per-cluster gradients (non-negative floats order
// like their bit patterns, so an unsigned max of the bits is the float max).
__global__ void __launch_bounds__(256) fixed_absmax(const float* gm, int64_t n, unsigned* absmax) {
  float m = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float a = fabsf(gm[i]);
    if (a <= 3.402823466e38f) m = fmaxf(m, a);  // finite values only
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) atomicMax(absmax, __float_as_uint(m));
}

// Exponent S of the fixed-point unit 2^-S: |g| < 2^e for the largest |g|, and
// n_hits terms of at most 2^(62 - cbits) each stay below 2^62.
__device__ __forceinline__ int fixed_shift(unsigned absmax_bits, int cbits) {
  int e = 0;
  frexpf(__uint_as_float(absmax_bits), &e);
  return 62 - cbits - e;
}

// Per block: a shared table of the 2 x 5472 fixed-point sums of the clusters
// the block visits, added into the global table at the end.
__global__ void __launch_bounds__(1024) fixed_accumulate(const float* gm, const uint16_t* rowsec, int n, int n_rows,
                                                         const unsigned* absmax, int cbits,
                                                         unsigned long long* table, unsigned* nonfinite) {
  extern __shared__ unsigned long long sh[];  // [kKeys * 2]
  for (int i = threadIdx.x; i < 2 * kKeys; i += blockDim.x) sh[i] = 0ull;
  __syncthreads();
  const int S = fixed_shift(*absmax, cbits);
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < n; h += gridDim.x * blockDim.x) {
    const int k = cluster_key(rowsec, h, n_rows);
    if (k == kKeyInvalid) continue;
    const float2 g = reinterpret_cast<const float2*>(gm)[h];
    if (!(fabsf(g.x) <= 3.402823466e38f) || !(fabsf(g.y) <= 3.402823466e38f)) {
      atomicOr(nonfinite + k, 1u);
      continue;
    }
    // g 2^S is exact in FP32 (|g 2^S| < 2^62) and rounds once to an integer
    const long long qx = __float2ll_rn(ldexpf(g.x, S));
    const long long qy = __float2ll_rn(ldexpf(g.y, S));
    atomicAdd(sh + 2 * k, (unsigned long long)qx);
    atomicAdd(sh + 2 * k + 1, (unsigned long long)qy);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * kKeys; i += blockDim.x)
    if (sh[i] != 0ull) atomicAdd(table + i, sh[i]);
}

// grad_align = -(sum) 2^-S, rounded once to FP32; NaN for a key with a
// non-finite cluster gradient.
__global__ void fixed_finish(const unsigned long long* table, const unsigned* nonfinite, const unsigned* absmax,
                             int cbits, float* grad_align) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * kKeys) return;
  const int S = fixed_shift(*absmax, cbits);
  const double v = ldexp((double)(long long)table[i], -S);
  grad_align[i] = nonfinite[i / 2] ? __int_as_float(0x7fc00000) : (float)(-v);
}

constexpr int kFixedThreads = 1024;
constexpr size_t kFixedSmem = sizeof(unsigned long long) * 2 * kKeys;  // 87,552 B

}  // namespace

size_t key_fixed_scratch_bytes() {
  return sizeof(unsigned long long) * 2 * kKeys + sizeof(unsigned) * (kKeys + 1);
}

cudaError_t launch_key_fixed_reduce(const float* grad_meas, const uint16_t* rowsec, int64_t n_hits, int n_rows,
                                    void* scratch, float* grad_align, cudaStream_t s) {
  static int blocks = 0;
  if (blocks == 0) {
    cudaError_t e = cudaFuncSetAttribute(fixed_accumulate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFixedSmem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fixed_accumulate, kFixedThreads, kFixedSmem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    blocks = sms * per_sm;
  }
  unsigned long long* table = static_cast<unsigned long long*>(scratch);
  unsigned* nonfinite = reinterpret_cast<unsigned*>(table + 2 * kKeys);
  unsigned* absmax = nonfinite + kKeys;
  cudaError_t e = cudaMemsetAsync(scratch, 0, key_fixed_scratch_bytes(), s);
  if (e != cudaSuccess || n_hits == 0) {
    if (e == cudaSuccess) e = cudaMemsetAsync(grad_align, 0, sizeof(float) * 2 * kKeys, s);
    return e;
  }
  int cbits = 0;
  while ((1ll << cbits) < n_hits + 1) ++cbits;
  const int n = (int)n_hits;
  const int nb = (int)(((int64_t)2 * n_hits + 255) / 256);
  fixed_absmax<<<nb < blocks * 8 ? nb : blocks * 8, 256, 0, s>>>(grad_meas, 2 * n_hits, absmax);
  const int na = (n + kFixedThreads - 1) / kFixedThreads;
  fixed_accumulate<<<na < blocks ? na : blocks, kFixedThreads, kFixedSmem, s>>>(grad_meas, rowsec, n, n_rows, absmax,
                                                                                   cbits, table, nonfinite);
  fixed_finish<<<(2 * kKeys + 255) / 256, 256, 0, s>>>(table, nonfinite, absmax, cbits, grad_align);
  return cudaGetLastError();
}

cudaError_t launch_key_reduce(const float* grad_meas, const int* sorted, const int* key_start, float* grad_align,
                              cudaStream_t s) {
  key_sum<<<(kKeys + 7) / 8, 256, 0, s>>>(grad_meas, sorted, key_start, grad_align);
  return cudaGetLastError();
}

}  // namespace tpcfit

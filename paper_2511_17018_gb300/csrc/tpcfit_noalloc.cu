// A fit entry point that allocates no device memory.
//
// Who needs it: code that runs where cudaMalloc / cudaFree must not be called,
// for instance a real-time loop that forbids allocator calls and the device
// synchronisation they can imply, or a host framework that hands out only the
// buffers it manages itself.  tpcfit_fit needs a handle, and creating one
// allocates (the alignment table, the error word, the length permutation);
// this entry point needs neither.  The time frame's constants travel in the
// launch's own argument block, as for every fit launch, so nothing is copied
// to the device for them.
//
// Its scratch (length histogram, work counter, error word, a zero alignment
// table and the length permutation) lives in one file-scope static device
// array of fixed size, which every GPU that loads the library keeps until the
// process exits.  The caller passes inputs and outputs as for tpcfit_fit.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "internal.h"
#include "tpcfit.h"

namespace tpcfit {
namespace {

// Scratch layout in 32-bit words.
constexpr int64_t kSortWords = 512;                              // length histogram + cursors
constexpr int64_t kWorkWords = 64;                               // work-item counter (+ padding)
constexpr int64_t kErrWords = 64;                                // error word (u64, 8-byte aligned)
constexpr int64_t kZeroAlignWords = kAlignFloats;                // never written: stays zero
constexpr int64_t kPermWords = TPCFIT_NOALLOC_MAX_TRACKS;        // length permutation
constexpr int64_t kOffSort = 0;
constexpr int64_t kOffWork = kOffSort + kSortWords;
constexpr int64_t kOffErr = kOffWork + kWorkWords;
constexpr int64_t kOffZeroAlign = kOffErr + kErrWords;
constexpr int64_t kOffPerm = (kOffZeroAlign + kZeroAlignWords + 63) / 64 * 64;
constexpr int64_t kScratchWords = kOffPerm + kPermWords;

static __device__ __align__(256) int32_t g_noalloc_scratch[kScratchWords];

// Device address of the scratch array, looked up once per device with that
// device current (in host code the array's name is only a host-side stand-in).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
int32_t* g_addr[kMaxDevices] = {};

cudaError_t scratch_address(int32_t** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<int32_t*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

}  // namespace
}  // namespace tpcfit

using namespace tpcfit;

extern "C" tpcfit_status tpcfit_fit_noalloc(const tpcfit_geometry* geometry, double bz_tesla, const float* alignment,
                                            int deterministic, const tpcfit_hits* hits, const int32_t* track_offsets,
                                            int32_t n_tracks, const float* seeds, float* params_out, float* cov_out,
                                            float* chi2_out, int32_t* ndf_out, void* stream) {
  if (!hits || n_tracks < 0 || hits->n_hits < 0 || (deterministic != 0 && deterministic != 1)) return TPCFIT_EINVAL;
  if (n_tracks > TPCFIT_NOALLOC_MAX_TRACKS) return TPCFIT_EINVAL;  // beyond the static scratch
  GeoConst geo;
  if (!build_geo(geometry, bz_tesla, geo)) return TPCFIT_EINVAL;
  if (n_tracks == 0) return TPCFIT_OK;
  if (!track_offsets || !seeds || !params_out || !cov_out || !chi2_out || !ndf_out) return TPCFIT_EINVAL;
  if (hits->n_hits > 0 && (!hits->y || !hits->z || !hits->rowsec)) return TPCFIT_EINVAL;
  if (hits->n_hits > INT32_MAX) return TPCFIT_EINVAL;
  if (!aligned(hits->y, 4) || !aligned(hits->z, 4) || !aligned(hits->rowsec, 2) || !aligned(track_offsets, 4) ||
      !aligned(seeds, 4) || !aligned(params_out, 4) || !aligned(cov_out, 4) || !aligned(chi2_out, 4) ||
      !aligned(ndf_out, 4) || (alignment && !aligned(alignment, 8)))
    return TPCFIT_EINVAL;
  int32_t* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) return TPCFIT_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* err = reinterpret_cast<unsigned long long*>(scratch + kOffErr);
  e = cudaMemsetAsync(err, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return TPCFIT_ECUDA;
  FitArgs a{};
  a.geo = geo;
  a.form = deterministic ? 0 : 1;  // the library's default factor
  a.y = hits->y;
  a.z = hits->z;
  a.rowsec = hits->rowsec;
  a.n_hits = hits->n_hits;
  a.off = track_offsets;
  a.n_tracks = n_tracks;
  a.seeds = seeds;
  a.align = alignment ? alignment : reinterpret_cast<const float*>(scratch + kOffZeroAlign);
  a.perm = scratch + kOffPerm;
  a.params = params_out;
  a.cov = cov_out;
  a.chi2 = chi2_out;
  a.ndf = ndf_out;
  a.err = err;
  a.work = reinterpret_cast<unsigned int*>(scratch + kOffWork);
  e = launch_length_order(track_offsets, n_tracks, scratch + kOffPerm, scratch + kOffSort, s);
  if (e != cudaSuccess) return TPCFIT_ECUDA;
  e = deterministic ? launch_fit_det(a, 1, 4, 24, s) : launch_fit_fast(a, 1, 4, 24, s);
  return e == cudaSuccess ? TPCFIT_OK : TPCFIT_ECUDA;
}

// Internal declarations shared by the host part of libtpcfit and its kernel
// modules.  Not part of the public C ABI (include/tpcfit.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "tpcfit.h"

namespace tpcfit {

constexpr int kNSectors = 36;
constexpr int kNSide = 18;
constexpr int kMaxRows = 152;
constexpr int kAlignFloats = kNSectors * kMaxRows * 2;
constexpr int kWarp = 32;
// The adjoint's checkpoints: the filter state before every kCkptEvery-th step
// of each pass, kCkptFloats floats each (p 5, L 25, x, sector bits, chi2, 3 pad).
constexpr int kCkptShift = 4;
constexpr int kCkptEvery = 1 << kCkptShift;
constexpr int kCkptFloats = 36;

// Per-time-frame constants of the fit, uploaded to the __constant__ bank of
// every kernel module (each compilation unit has its own copy, Sec. 4.1).
struct GeoConst {
  float row_x[kMaxRows];      // local x of each pad-row plane (FP64 -> FP32)
  float rot_c[kNSide * kNSide];  // cos / sin of the rotation from sector a to b
  float rot_s[kNSide * kNSide];  //   (index a * 18 + b), FP64 -> FP32
  double asin_a[30];          // Maclaurin coefficients of arcsin (FP64 island)
  float kappa;                // -0.00299792458 * Bz  [1/cm per (c/GeV)]
  float v_meas;               // cluster variance (0.1 cm)^2
  float sqrt_v;               // its square root (fast-mode Potter coefficients)
  float l0;                   // sqrt of the initial covariance diagonal (10)
  float max_snp;              // |sin phi| limit (0.999)
  int32_t n_rows;
};

// Arguments of one fit launch.
struct FitArgs {
  const float* y;
  const float* z;
  const uint16_t* rowsec;
  int64_t n_hits;
  const int32_t* off;
  int32_t n_tracks;
  const float* seeds;
  const float* align;          // [36][152][2], always valid (zeros when unset)
  const int32_t* perm;         // [n_tracks] processing order, or null
  float* params;
  float* cov;
  float* chi2;
  int32_t* ndf;
  unsigned long long* err;     // error word: code << 56 | track
  unsigned int* work;          // work-item counter (zeroed by the launcher)
  // checkpoint recording for the adjoint (null = off)
  float* ck;                   // [2][ck_slots][36] filter state before every kCkptEvery-th step of each pass
  int32_t* ck_last;            // [n_tracks] index of the last cluster of the outward pass
  int64_t ck_slots;            // slots per pass: n_hits / kCkptEvery + n_tracks + 1
  // several time frames in one launch (frame_base = null: one frame)
  const int64_t* frame_base;   // [n_frames + 1] first track of each frame
  int32_t n_frames;
  const float* frame_align;    // [n_frames][36][152][2] per-frame offsets, or null (handle's table)
  const int32_t* frame_ready;  // [n_frames] ready flags (!= 0 when the frame's clusters are in place), or null
  int64_t wait_ns;             // bound of a ready-flag wait
};

// Arguments of one backward launch (same frame as the recorded fit).
struct BwdArgs {
  const float* y;
  const float* z;
  const uint16_t* rowsec;
  int64_t n_hits;
  const int32_t* off;
  int32_t n_tracks;
  const float* align;
  const int32_t* perm;
  const int32_t* ndf;          // outputs of the recorded fit
  const float* ck;
  const int32_t* ck_last;
  int64_t ck_slots;
  const float* grad_chi2;      // [n_tracks] dL/dchi2_i
  float* grad_seeds;           // [5][n_tracks]
  float* grad_meas;            // [n_hits][2] dL/dm per cluster, or null
  float* grad_align_atomic;    // [36][152][2] accumulated with atomics, or null
  unsigned int* work;
  float4* seg;                 // segment store: [resident warps][kCkptEvery][8][32] float4
};

// Error codes recorded in the device error word.
constexpr unsigned long long kErrOffsets = 1;
constexpr unsigned long long kErrRowSector = 2;
constexpr unsigned long long kErrTimeout = 3;

// ---- constant-memory registry (Sec. 4.1): every kernel module registers an
// uploader for its own __constant__ copy; the host updates all of them.
using ConstUploader = cudaError_t (*)(const GeoConst&, cudaStream_t);
struct ConstRegistration {
  ConstRegistration(const char* module, ConstUploader up);
};
cudaError_t upload_constants_all(const GeoConst& g, cudaStream_t s);
void forget_resident_constants();
int registered_constant_modules();

// Geometry and field -> per-time-frame constants (host, FP64 rounded to FP32);
// false for an invalid geometry.
bool build_geo(const tpcfit_geometry* g, double bz, GeoConst& out);

// ---- kernel launchers, one per module
cudaError_t launch_fit_fast(const FitArgs& a, int lanes_per_track, int rows_per_stage, int warps, cudaStream_t s);
cudaError_t launch_fit_det(const FitArgs& a, int lanes_per_track, int rows_per_stage, int warps, cudaStream_t s);
cudaError_t launch_backward_fast(const BwdArgs& a, int warps, cudaStream_t s);
cudaError_t launch_backward_det(const BwdArgs& a, int warps, cudaStream_t s);
// float4 elements of the segment store a backward launch with `warps` needs
cudaError_t backward_store_fast(int warps, int64_t& float4s);
cudaError_t backward_store_det(int warps, int64_t& float4s);
// true if `warps` is a compiled backward block shape
bool backward_shape_supported(int warps);

// Deterministic per-key reduction of cluster gradients (key_reduce.cu).
size_t key_sort_scratch_bytes(int64_t n_hits);
cudaError_t launch_key_sort(const uint16_t* rowsec, int64_t n_hits, int n_rows, void* scratch, int** sorted_out,
                            int** key_start_out, cudaStream_t s);
cudaError_t launch_key_reduce(const float* grad_meas, const int* sorted, const int* key_start, float* grad_align,
                              cudaStream_t s);
// true if (lanes_per_track, rows_per_stage, warps) is a compiled launch shape
bool fit_shape_supported(int lanes_per_track, int rows_per_stage, int warps);

// Ordering by (frame ascending, length descending) for batched frames.
// scratch: int32 [2 * n_frames * 256 + scan_tmp_ints(n_frames * 256)].
int64_t frame_order_scratch_ints(int32_t n_frames);
cudaError_t launch_frame_length_order(const int32_t* off, int32_t n_tracks, const int64_t* frame_base,
                                      int32_t n_frames, int32_t* perm, int32_t* scratch, cudaStream_t s);
// Exclusive prefix sum of n ints in place (key_reduce.cu); tmp: scan_tmp_ints(n) ints.
int64_t scan_tmp_ints(int64_t n);
cudaError_t launch_scan_exclusive(int* v, int n, int* tmp, cudaStream_t s);

// Length-ordering permutation: perm[k] = track processed k-th, longest first.
// scratch: int32[2 * 256] (zeroed by the launcher).
cudaError_t launch_length_order(const int32_t* off, int32_t n_tracks, int32_t* perm, int32_t* scratch,
                                cudaStream_t s);

}  // namespace tpcfit

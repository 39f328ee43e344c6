// Internal declarations shared by the host part of libtpcfit and its kernel
// modules.  Not part of the public C ABI (include/tpcfit.h).
#pragma once

#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "kernel_abi.h"
#include "tpcfit.h"

namespace tpcfit {

// Geometry and field -> per-time-frame constants (host, FP64 rounded to FP32);
// false for an invalid geometry.
bool build_geo(const tpcfit_geometry* g, double bz, GeoConst& out);

// ---- kernel launchers, one per module
cudaError_t launch_fit_fast(const FitArgs& a, int lanes_per_track, int rows_per_stage, int warps, cudaStream_t s);
cudaError_t launch_fit_det(const FitArgs& a, int lanes_per_track, int rows_per_stage, int warps, cudaStream_t s);
cudaError_t launch_backward_fast(const BwdArgs& a, int warps, cudaStream_t s);
cudaError_t launch_backward_det(const BwdArgs& a, int warps, cudaStream_t s);
// float4 elements of the segment store a fast backward launch without material
// with `warps`, the physics bits phys and the factor form (0 square root, 1 U-D)
// needs
cudaError_t backward_store_fast(int warps, int phys, int form, int64_t& float4s);
// float4 elements of the backward's tape for n_tracks tracks
int64_t backward_tape_float4s(int64_t n_tracks);
// the two-filter smoother of a recorded fit, and its segment store (float4s)
cudaError_t launch_smooth_fast(const SmoothArgs& a, cudaStream_t s);
cudaError_t launch_smooth_det(const SmoothArgs& a, cudaStream_t s);
cudaError_t smooth_store_fast(int64_t& float4s);
cudaError_t smooth_store_det(int64_t& float4s);
// true if `warps` is a compiled backward block shape
bool backward_shape_supported(int warps);

// Deterministic per-key reduction of cluster gradients (key_reduce.cu).
size_t key_sort_scratch_bytes(int64_t n_hits);
cudaError_t launch_key_sort(const uint16_t* rowsec, int64_t n_hits, int n_rows, void* scratch, int** sorted_out,
                            int** key_start_out, cudaStream_t s);
cudaError_t launch_key_reduce(const float* grad_meas, const int* sorted, const int* key_start, float* grad_align,
                              cudaStream_t s);
// The order-independent alternative: fixed-point integer sums per key (the
// deterministic mode's default); scratch of key_fixed_scratch_bytes().
size_t key_fixed_scratch_bytes();
cudaError_t launch_key_fixed_reduce(const float* grad_meas, const uint16_t* rowsec, int64_t n_hits, int n_rows,
                                    void* scratch, float* grad_align, cudaStream_t s);
// true if (lanes_per_track, rows_per_stage, warps) is a compiled launch shape
bool fit_shape_supported(int lanes_per_track, int rows_per_stage, int warps);

// ---- run-time compilation of the fit (rtc.cpp, Sec. 5)
bool rtc_available();
long long rtc_compile_count();
const char* rtc_log();
// The NVRTC source of the fit for these constants and mode.
std::string rtc_fit_source(const GeoConst& g, bool det);
// NVRTC only (no device needed): the CUBIN of a variant, stored in cache_dir
// when given.
tpcfit_status rtc_build(const GeoConst& g, bool det, int rps, int warps, bool record, bool frames,
                        const char* cache_dir);
// Compile (once per source and variant) and launch the fit specialised for g.
tpcfit_status rtc_launch_fit(const GeoConst& g, bool det, int rps, int warps, const FitArgs& a, const char* cache_dir,
                             cudaStream_t s);

// Ordering by (frame ascending, length descending) for batched frames.
// scratch: int32 [2 * n_frames * 256 + scan_tmp_ints(n_frames * 256)].
int64_t frame_order_scratch_ints(int32_t n_frames);
cudaError_t launch_frame_length_order(const int32_t* off, int32_t n_tracks, const int64_t* frame_base,
                                      int32_t n_frames, int32_t* perm, int32_t* scratch, cudaStream_t s);
// Outlier rejection (reject.cu): the clusters with chi2 > cut dropped, the
// others copied in order; off_out [n_tracks + 1] receives the new offsets.
// scratch: reject_scratch_ints(n_tracks) ints.
int64_t reject_scratch_ints(int32_t n_tracks);
cudaError_t launch_reject(const int32_t* off, int32_t n_tracks, const float* y, const float* z, const uint16_t* rowsec,
                          int64_t n_hits, const float* chi2, float cut, float* y_out, float* z_out,
                          uint16_t* rowsec_out, int32_t* off_out, int32_t* scratch, cudaStream_t s);
// Exclusive prefix sum of n ints in place (key_reduce.cu); tmp: scan_tmp_ints(n) ints.
int64_t scan_tmp_ints(int64_t n);
cudaError_t launch_scan_exclusive(int* v, int n, int* tmp, cudaStream_t s);

// Length-ordering permutation: perm[k] = track processed k-th, longest first.
// scratch: int32[2 * 256] (zeroed by the launcher).
cudaError_t launch_length_order(const int32_t* off, int32_t n_tracks, int32_t* perm, int32_t* scratch,
                                cudaStream_t s);

}  // namespace tpcfit

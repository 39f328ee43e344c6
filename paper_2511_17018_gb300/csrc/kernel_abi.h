// Layouts shared by the host part of libtpcfit, its ahead-of-time kernel
// modules and the fit compiled at run time (Sec. 5).  Compiles under nvcc,
// the host compiler and NVRTC (which provides no standard headers).
#pragma once

#ifdef __CUDACC_RTC__
typedef signed char int8_t;
typedef short int16_t;
typedef int int32_t;
typedef long long int64_t;
typedef unsigned char uint8_t;
typedef unsigned short uint16_t;
typedef unsigned int uint32_t;
typedef unsigned long long uint64_t;
typedef unsigned long long uintptr_t;
#else
#include <cstdint>
#include <cuda_runtime.h>
#endif

namespace tpcfit {

constexpr int kNSectors = 36;
constexpr int kNSide = 18;
constexpr int kMaxRows = 152;
constexpr int kAlignFloats = kNSectors * kMaxRows * 2;
constexpr int kWarp = 32;
// The adjoint's checkpoints: the filter state before every kCkptEvery-th step
// of each pass, kCkptFloats floats each (p 5, L 25, x, sector bits: what the
// recomputation starts from; chi2 is not needed, since only the inward pass's
// total enters the objective and its adjoint is a constant).
constexpr int kCkptShift = 4;
constexpr int kCkptEvery = 1 << kCkptShift;
constexpr int kCkptFloats = 32;

// Per-time-frame constants of the fit (Sec. 4.1).  Every launch carries them
// by value in its argument block, i.e. in the kernel-parameter constant bank
// (3.4 KB of the 32 KB a launch may pass), so launches of different handles
// and replays of captured graphs never share or overwrite them.
struct GeoConst {
  float row_x[kMaxRows];      // local x of each pad-row plane (FP64 -> FP32)
  float rot_c[kNSide * kNSide];  // cos / sin of the rotation from sector a to b
  float rot_s[kNSide * kNSide];  //   (index a * 18 + b), FP64 -> FP32
  float kappa;                // -0.00299792458 * Bz  [1/cm per (c/GeV)]
  float v_meas;               // cluster variance (0.1 cm)^2
  float sqrt_v;               // its square root (fast-mode Potter coefficients)
  float l0;                   // sqrt of the initial covariance diagonal (10)
  float max_snp;              // |sin phi| limit (0.999)
  int32_t n_rows;
  // a thin material layer at every pad row (mat = 0: none)
  int32_t mat;
  float x0_inv;               // 1 / radiation length [1/cm]
  float dedx;                 // minimum-ionising energy loss [GeV/cm]
  float mass2;                // particle mass squared [GeV^2]
  float d_row;                // layer thickness at normal incidence [cm]
  // field map Bz(r, z) = Bz0 (1 + c_r (r / 250)^2 + c_z (z / 250)^2) (field = 0: uniform)
  int32_t field;
  float f_r, f_z;             // c_r / 250^2, c_z / 250^2 [1/cm^2]
};

// Arguments of one fit launch.
struct FitArgs {
  GeoConst geo;                // the time frame's constants
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
  float* ck;                   // [2][ck_slots][32] filter state before every kCkptEvery-th step of each pass
  int32_t* ck_last;            // [n_tracks] index of the last cluster of the outward pass
  int64_t ck_slots;            // slots per pass: n_hits / kCkptEvery + n_tracks + 1
  // several time frames in one launch (frame_base = null: one frame)
  const int64_t* frame_base;   // [n_frames + 1] first track of each frame
  int32_t n_frames;
  const float* frame_align;    // [n_frames][36][152][2] per-frame offsets, or null (handle's table)
  const int32_t* frame_ready;  // [n_frames] ready flags (!= 0 when the frame's clusters are in place), or null
  int64_t wait_ns;             // bound of a ready-flag wait
  int32_t mat;                 // material layers on (selects the kernel variant that crosses them)
  int32_t field;               // field map on (selects the kernel variant that follows it)
  int32_t form;                // factor of the covariance: 0 square root (L), 1 U-D (fast mode without material)
};

// Arguments of one backward launch (same frame as the recorded fit).
struct BwdArgs {
  GeoConst geo;
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
  float4* tape;                // or the tape: [2][n_hits][8] float4, the state before every step (null: segment store)
  int32_t phys;                // physics of the recorded fit: bit 1 material layers, bit 2 the field map
  int32_t form;                // factor the fast one-kernel backward recomputes in: 0 square root (L), 1 U-D
  int32_t ck_form;             // factor the checkpoints hold: 0 L, 1 U-D (u, d)
};

// Arguments of one smoother launch (same frame as the recorded fit).
struct SmoothArgs {
  GeoConst geo;
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
  float* resid;                // [n_hits][2] m - H x_u
  float* rcov;                 // [n_hits][3] R00, R10, R11 of V + H C_u H^T
  float* chi2;                 // [n_hits] r^T R^-1 r
  float* state;                // [n_hits][5] smoothed state from all clusters, or null
  float* state_cov;            // [n_hits][15] its covariance (packed)
  unsigned int* work;
  float4* seg;                 // segment store, as for the adjoint
  int32_t ck_form;             // factor the checkpoints hold: 0 L, 1 U-D (u, d)
  int32_t mat;                 // material layers on (the recorded fit had them)
};

// Error codes recorded in the device error word.
constexpr unsigned long long kErrOffsets = 1;
constexpr unsigned long long kErrRowSector = 2;
constexpr unsigned long long kErrTimeout = 3;

// Shared memory of a fit block (geometry tables + alignment table) and of one
// warp's double-buffered cluster staging with `rps` clusters per refill: the
// host sizes the launch of a kernel compiled at run time with these.
constexpr int kTablesFloats = kMaxRows + 2 * kNSide * kNSide;
constexpr int kFitBlockSmemBytes = 4 * (kTablesFloats + kAlignFloats);
__host__ __device__ constexpr int fit_warp_stage_bytes(int rps) { return 3 * 2 * kWarp * (rps + 1) * 4; }
// Blocks per SM the fit asks for (__launch_bounds__) at each supported shape.
__host__ __device__ constexpr int fit_min_blocks(int rps, int warps) { return (rps == 4 && warps == 24) || rps == 16 || warps == 16 ? 1 : 2; }

}  // namespace tpcfit

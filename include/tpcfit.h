/*
 * tpcfit -- batched Kalman fit of TPC track candidates on one GB300 GPU.
 *
 * The operation: every track candidate of a time frame (its clusters, at most
 * one per pad row, ordered by row) is fitted as a helix in a uniform Bz field.
 * The track state is propagated from pad row to pad row in the local frame of
 * its TPC sector, rotated into the next sector's frame when the candidate
 * crosses a sector boundary, and updated with each 2D cluster (y, z) while
 * chi2 accumulates.  The fit consists of an outward pass from the seed and an
 * inward refit.  Source: the paper names track propagation through the
 * magnetic field as the shared component of TPC tracking (Sec. 4) and the time
 * frame as the processing unit (Sec. 1).  The deterministic mode follows the
 * rules of Sec. 2; the per-time-frame constants of Sec. 4.1 travel with
 * every kernel launch in its argument block (the kernel-parameter constant
 * bank), so handles never share them.
 *
 * Conventions (all calls):
 *   - Units cm, GeV/c, T.  Track state p = (y, z, sin phi, tan lambda, q/pt)
 *     at local x = X_row, in the frame of a sector; the covariance is packed
 *     lower-triangular: (00, 10, 11, 20, 21, 22, 30, 31, 32, 33, 40, .., 44).
 *   - Sectors 0-17 are the A side (z >= 0), 18-35 the C side, sector s centred
 *     at azimuth ((s mod 18) + 0.5) * sector_width.  rowsec = row << 6 | sector.
 *   - Arrays are structure-of-arrays: params_out[5][n_tracks] means component
 *     c of track i at params_out[c * n_tracks + i].
 *   - "device" pointers must be CUDA device memory of the current device;
 *     "host" pointers ordinary host memory.  The library never frees caller
 *     memory and keeps no pointer to it after a call returns, except where a
 *     call says otherwise.
 *   - stream is a cudaStream_t (NULL = the legacy default stream).  Every call
 *     that takes a stream only enqueues work on it and returns; argument
 *     errors are returned synchronously before anything is enqueued.
 *   - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef TPCFIT_H_
#define TPCFIT_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TPCFIT_OK = 0,
  TPCFIT_EINVAL = 1,   /* bad argument (null pointer, negative or inconsistent size) */
  TPCFIT_ECUDA = 2,    /* a CUDA runtime call failed */
  TPCFIT_ENOMEM = 3,   /* device allocation failed */
  TPCFIT_EDEVICE = 4,  /* a kernel found invalid input (see tpcfit_get_status) */
  TPCFIT_ETIMEOUT = 5, /* a bounded device-side wait ran out */
  TPCFIT_ESTATE = 6,   /* call not allowed in the handle's current state */
  TPCFIT_ERTC = 7      /* run-time compilation unavailable or failed (see tpcfit_rtc_log) */
} tpcfit_status;

/* Detector geometry (copied at tpcfit_create; row_x is a host array). */
typedef struct {
  int32_t n_sectors;       /* must be 36 */
  int32_t n_rows;          /* 1..152 */
  const double* row_x;     /* host [n_rows]: local x of each pad-row plane, cm, ascending */
  double sector_width_deg; /* must be 20: 18 sectors per side cover the circle */
  double z_max;            /* 250 cm (informational) */
} tpcfit_geometry;

/* Clusters of a time frame, device SoA, track-major (a track's clusters are
 * contiguous and ordered by increasing row). */
typedef struct {
  const float* y;          /* device [n_hits] local y, cm */
  const float* z;          /* device [n_hits] z, cm */
  const uint16_t* rowsec;  /* device [n_hits] row << 6 | sector */
  int64_t n_hits;
} tpcfit_hits;

typedef struct tpcfit_handle tpcfit_handle;

/* Create a fitter on the current CUDA device for the given geometry and field.
 * Builds the geometry tables (pad-row x, sector rotation cos/sin) on the host in
 * FP64 and rounds them to FP32; the handle keeps them and passes them to every
 * kernel it launches.  Returns EINVAL for a bad geometry, ECUDA/ENOMEM on CUDA
 * failure. */
tpcfit_status tpcfit_create(const tpcfit_geometry* geometry, double bz_tesla, tpcfit_handle** out);

/* Release the handle and its device scratch.  Synchronises the device first.
 * NULL is ignored. */
void tpcfit_destroy(tpcfit_handle* h);

/* Run-time switch between the fast FP32 mode (0, default: FMA contraction,
 * approximate division and square root) and the deterministic mode (1: IEEE
 * FP32 without contraction, fixed operation order, results bit-identical to the
 * strict-FP32 host reference and independent of launch configuration), as the
 * run-time part of the deterministic mode of Sec. 2. */
tpcfit_status tpcfit_set_mode(tpcfit_handle* h, int deterministic);

/* Launch configuration of the fit: lanes_per_track (1 = one track per lane),
 * rows_per_stage (clusters per track staged into shared memory per refill) and
 * warps_per_block.  Supported (rows_per_stage, warps_per_block) shapes:
 * (4, 8), (4, 12), (4, 24), (8, 8), (8, 16), (16, 8); default (4, 24).
 * sort_by_length != 0 (default) orders tracks by length before the fit so that
 * a warp's tracks finish together.  In deterministic mode the results do not
 * depend on these choices.  EINVAL for unsupported values. */
tpcfit_status tpcfit_set_config(tpcfit_handle* h, int lanes_per_track, int rows_per_stage, int warps_per_block,
                                int sort_by_length);

/* Alignment offsets d[36][152][2] (dy, dz per sector and row, cm) subtracted
 * from every cluster before the fit.  d is a device pointer; its contents are
 * copied into the handle on `stream` (so the caller may overwrite d after the
 * copy has run).  d = NULL sets all offsets to zero.  Offsets are constant per
 * time frame, like the calibration constants of Sec. 4.1. */
tpcfit_status tpcfit_set_alignment(tpcfit_handle* h, const float* d, void* stream);

/* Pre-size the handle's device scratch for up to max_tracks tracks (the length
 * permutation) so that later fits allocate nothing, e.g. during CUDA-graph
 * capture.  Synchronous. */
tpcfit_status tpcfit_reserve(tpcfit_handle* h, int64_t max_tracks, int64_t max_hits);

/* Fit n_tracks tracks.
 *   track_offsets: device int32 [n_tracks + 1], non-decreasing, offsets into the
 *                  hit arrays; track i owns hits [off[i], off[i+1]).
 *   seeds:         device float [5][n_tracks], state at the track's first hit.
 *   params_out:    device float [5][n_tracks]  inward-refit state at the first hit
 *                  (x = X of that hit's row, frame of that hit's sector);
 *   cov_out:       device float [15][n_tracks] its covariance (packed);
 *   chi2_out:      device float [n_tracks]     chi2 of the inward refit;
 *   ndf_out:       device int32 [n_tracks]     2 * clusters used - 5.
 * A track whose fit fails numerically (|sin phi| >= 0.999, a backward step
 * through a sector rotation, fewer than 3 clusters) is not an error: it gets
 * ndf = -1 and NaN parameters, covariance and chi2.  A track with invalid input
 * (offsets out of order or beyond n_hits, row >= n_rows, sector >= 36) gets
 * ndf = -2 and NaNs, and the handle's error word records it (tpcfit_get_status).
 * n_tracks = 0 is a no-op.  May allocate scratch (see tpcfit_reserve). */
tpcfit_status tpcfit_fit(tpcfit_handle* h, const tpcfit_hits* hits, const int32_t* track_offsets, int32_t n_tracks,
                         const float* seeds, float* params_out, float* cov_out, float* chi2_out, int32_t* ndf_out,
                         void* stream);

/* Fit many time frames in one persistent launch.  The clusters, offsets,
 * seeds and outputs of all frames are concatenated (track-major, as for
 * tpcfit_fit with n_tracks tracks in total); frame f owns tracks
 * [frame_track_base[f], frame_track_base[f + 1]) (device int64 [n_frames + 1],
 * frame_track_base[0] = 0, frame_track_base[n_frames] = n_tracks).
 *   frame_alignment: device float [n_frames][36][152][2], the per-frame offsets
 *                    (constants that change between time frames, Sec. 4.1), or
 *                    NULL to use the handle's alignment for every frame.
 *   frame_ready:     device int32 [n_frames] flags, or NULL.  With flags, warps
 *                    wait (acquire load, polled) until the flag of each of their
 *                    tracks' frames is nonzero before reading its clusters, so the
 *                    caller may copy frames in on another stream and set each flag
 *                    after its frame's copy.  A wait gives up after
 *                    wait_timeout_ns of device time (0 = 1 s): the frame's tracks
 *                    get ndf = -3 and tpcfit_get_status returns ETIMEOUT.  With
 *                    flags, `stream` must not be the legacy default stream (NULL),
 *                    whose implicit ordering would hold the copies back (EINVAL).
 * Work is ordered by frame, then by decreasing track length.  Recording for
 * the adjoint does not apply (tpcfit_fit_backward returns ESTATE after this).
 * Capturable in a CUDA graph after one call with the same sizes has run
 * outside the capture (scratch is then in place); the captured launches hold
 * the handle's constants as they were at capture. */
tpcfit_status tpcfit_fit_frames(tpcfit_handle* h, const tpcfit_hits* hits, const int32_t* track_offsets,
                                int32_t n_tracks, const int64_t* frame_track_base, int32_t n_frames,
                                const float* frame_alignment, const int32_t* frame_ready, int64_t wait_timeout_ns,
                                const float* seeds, float* params_out, float* cov_out, float* chi2_out,
                                int32_t* ndf_out, void* stream);

/* Material correction (Sec. 4: the material budget is part of the shared
 * propagation): a thin layer at every pad row, of radiation length x0_cm,
 * minimum-ionising energy loss dedx_gev_cm and thickness row_cm at normal
 * incidence, for a particle of mass mass_gev.  The state at a row is the one
 * the track leaves it with; the outward pass crosses a row's layer on
 * arriving, the inward pass undoes it before leaving the row.  A layer is
 * crossed over l = row_cm sqrt(1 + tan^2 lambda) / cos phi; the energy drops by
 * dedx l / beta^2 and the direction scatters with the Highland angle (without
 * its logarithmic term), added as process noise.  x0_cm <= 0: no material
 * (default).  The fit, the smoother, the batched and run-time-compiled fits
 * and tpcfit_fit_backward follow it (the backward in its 8-warp shape,
 * whatever tpcfit_set_backward_config chose).  EINVAL for non-finite or
 * non-positive values. */
tpcfit_status tpcfit_set_material(tpcfit_handle* h, double x0_cm, double dedx_gev_cm, double mass_gev, double row_cm);

/* Non-uniform field (Sec. 4: propagation through the magnetic field): the
 * analytic map Bz(r, z) = bz_tesla (1 + c_r (r / 250 cm)^2 + c_z (z / 250 cm)^2)
 * (bz_tesla from tpcfit_create).  Each step is a helix with Bz at the step's
 * midpoint, estimated by a straight half step from its start; the Jacobian
 * treats the step's curvature as constant.  c_r = c_z = 0: uniform (default).
 * The fit, the smoother and the batched and run-time-compiled fits follow it,
 * and so does tpcfit_fit_backward: its reverse runs through the midpoint
 * curvature (in its 8-warp shape, whatever tpcfit_set_backward_config chose).
 * EINVAL for non-finite values. */
tpcfit_status tpcfit_set_field_map(tpcfit_handle* h, double c_r, double c_z);

/* Run-time compilation of the fit (Sec. 5).  enable = 1: tpcfit_fit and
 * tpcfit_fit_frames run a fit kernel compiled with NVRTC for this handle's
 * geometry, field, mode and launch shape, in which those per-time-frame values
 * are compile-time constants.  Each variant (constants, mode, shape, recording,
 * batched frames) is compiled on its first use, which takes about a second,
 * and kept for the life of the process; with cache_dir (NULL: none) its CUBIN
 * is also kept in that directory for later processes.  The first fit of a
 * variant therefore belongs outside stream capture.  The device code is the
 * one compiled ahead of time, with the same flags: deterministic results are
 * bit-identical to the ahead-of-time kernels, fast-mode results are within the
 * fast-mode tolerance.  enable = 0 (default): ahead-of-time kernels.  ERTC if
 * NVRTC cannot be loaded; a failed compilation or load reports ERTC / ECUDA
 * from the fit. */
tpcfit_status tpcfit_set_rtc(tpcfit_handle* h, int enable, const char* cache_dir);

/* Compile one fit variant with NVRTC and store its CUBIN in cache_dir (NULL:
 * compile only), without a device: fills the cache before a run.  Arguments as
 * for tpcfit_create, tpcfit_set_mode, tpcfit_set_config and tpcfit_set_record;
 * frames != 0 for the batched-frame variant.  EINVAL for an invalid geometry
 * or shape, ERTC if NVRTC is missing or the compilation fails. */
tpcfit_status tpcfit_rtc_build(const tpcfit_geometry* geometry, double bz_tesla, int deterministic, int rows_per_stage,
                               int warps_per_block, int record, int frames, const char* cache_dir);

/* 1 if NVRTC can be loaded in this process. */
int tpcfit_rtc_available(void);
/* NVRTC compilations this process has run (cache hits do not count). */
long long tpcfit_rtc_compile_count(void);
/* Log of the last NVRTC compilation (empty if none); valid until the next one. */
const char* tpcfit_rtc_log(void);

/* Record checkpoints for the adjoint (record = 1) or not (0, default).  With
 * recording on, tpcfit_fit also stores the filter state before every 16th step
 * of both passes (about 8 floats per cluster, handle-owned, grown as needed) so
 * that tpcfit_fit_backward can follow.  Any tpcfit_fit call replaces the
 * recording. */
tpcfit_status tpcfit_set_record(tpcfit_handle* h, int record);

/* Launch configuration of the adjoint's reverse: warps per block (4, 8, 10 or
 * 12; default 8).  Each resident warp owns 8-12 KB of shared memory that holds
 * the states it copies ahead (and, in fast mode without material, a segment
 * store in device memory that the handle allocates on the first backward).
 * Results do not depend on it.  EINVAL for other values. */
tpcfit_status tpcfit_set_backward_config(tpcfit_handle* h, int warps_per_block);

/* Factor of the covariance that the fast fit without material layers carries:
 * 1 = U-D (C = U D U^T, Bierman's measurement updates, modified weighted
 * Gram-Schmidt at sector rotations; default), 0 = the square-root factor
 * (C = L L^T, Potter's updates).  Both compute the same extended Kalman filter
 * and differ in FP32 rounding and speed; the deterministic mode and the
 * material layers always take the square-root factor (its strict-FP32
 * sequence is the deterministic mode's reference).  The recording keeps the
 * factor of the form the fit ran in; the smoother and the backward read
 * either.  The paper prescribes no factorisation; this is an implementation
 * choice.  Replaces the recording.
 * EINVAL for other values. */
tpcfit_status tpcfit_set_fit_form(tpcfit_handle* h, int form);

/* Factor of the covariance that the fast backward without material layers
 * recomputes its segments in: 1 = U-D (C = U D U^T, U unit upper triangular,
 * Bierman's measurement updates; default), 0 = the square-root factor
 * (C = L L^T, Potter's updates).  Both give the gradient of the same fit; they
 * differ in FP32 rounding and speed (U-D: 15 factor entries instead of 25, 6
 * float4 per stored state instead of 8).  The square-root reverse needs a
 * recording made in the square-root form (tpcfit_set_fit_form 0, or one lane
 * per track not in effect): its adjoint crosses segment boundaries only if the
 * recomputed factor is the recorded one; after a U-D fit tpcfit_fit_backward
 * answers ESTATE in that form.  The paper prescribes no factor for the
 * adjoint; this is an implementation choice.  The deterministic mode and the
 * material layers always take the square-root factor.  EINVAL for other
 * values. */
tpcfit_status tpcfit_set_backward_form(tpcfit_handle* h, int form);

/* How the deterministic mode sums the per-cluster gradients into grad_align
 * (Sec. 2 asks for results that do not depend on the order of parallel work):
 *   0 (default): each cluster gradient is rounded once to a 64-bit
 *     fixed-point integer with the unit 2^-S, S fixed per call by the largest
 *     finite |gradient| and the cluster count so that no sum can overflow;
 *     integer addition does not depend on its order, and each key's sum is
 *     rounded once to FP32 (NaN where a cluster gradient is not finite);
 *   1: the clusters are sorted by (sector, row) with a stable radix sort and
 *     each key is summed in FP32 in a fixed order.
 * Both give the same bits in every run and launch shape; 0 is the closer to
 * the exact sum (its only rounding: 2^-S per cluster, at most about 1e-11 of
 * the largest gradient at 400,000 tracks, and the final FP32 rounding) and
 * the faster.  Fast mode is not affected.  EINVAL for other values. */
tpcfit_status tpcfit_set_det_reduction(tpcfit_handle* h, int method);

/* Adjoint of the recorded fit: gradients of L = sum_i grad_chi2[i] * chi2_i.
 * Inputs must be those of the last tpcfit_fit on this handle, which must have
 * run with recording on and in the same mode, and, for the square-root
 * reverse (tpcfit_set_backward_form 0), in the square-root form (otherwise
 * ESTATE):
 *   hits, track_offsets, n_tracks: as for tpcfit_fit;
 *   ndf:        device int32 [n_tracks], the ndf output of that fit;
 *   grad_chi2:  device float [n_tracks], dL/dchi2_i.
 * Outputs (device, overwritten):
 *   grad_align: float [36][152][2], dL/d(dy, dz) of the alignment offsets;
 *   grad_seeds: float [5][n_tracks], dL/dseed;
 *   grad_meas:  float [n_hits][2], dL/d(measured y, z) per cluster, or NULL.
 * The backward recomputes each 16-step segment from its checkpoint and runs
 * the hand-written reverse of every step, copying the state before each step
 * into shared memory one step ahead.  Fast mode without material layers
 * recomputes into a per-warp segment store in the same kernel, in the factor
 * form tpcfit_set_backward_form chose; the
 * deterministic mode and the material layers replay the segments in a kernel
 * of their own onto a tape of every step's state (about 40 MB per 1,000
 * tracks, handle-owned, grown as needed) and reverse from it.  It follows the
 * field map and the material layers (tpcfit_set_field_map,
 * tpcfit_set_material).  Tracks of more than 152 clusters get no gradient in
 * the taped cases.  Fast mode accumulates grad_align with
 * atomics; deterministic mode writes per-cluster gradients and reduces them
 * per (sector, row) so that grad_align is bitwise reproducible, by the method
 * tpcfit_set_det_reduction chose.  Tracks with ndf <= 0 contribute 0. */
tpcfit_status tpcfit_fit_backward(tpcfit_handle* h, const tpcfit_hits* hits, const int32_t* track_offsets,
                                  int32_t n_tracks, const int32_t* ndf, const float* grad_chi2, float* grad_align,
                                  float* grad_seeds, float* grad_meas, void* stream);

/* Two-filter smoother of the recorded fit: for every cluster, the residual
 * against the estimate from all the other clusters of its track (the outward
 * prediction from the seed and the clusters before it, combined with the
 * inward prediction from the clusters after it).  Inputs as for
 * tpcfit_fit_backward (the last tpcfit_fit on this handle, with recording on,
 * same mode; otherwise ESTATE).  Outputs (device, overwritten):
 *   resid: float [n_hits][2], measured (y, z) minus alignment minus the
 *          smoothed (y, z);
 *   rcov:  float [n_hits][3], (R00, R10, R11) of R = V + H C H^T;
 *   chi2:  float [n_hits], resid^T R^-1 resid (2 degrees of freedom), the
 *          outlier test of the cluster.
 * NaN for the clusters of tracks with ndf <= 0 and for clusters the outward
 * pass did not reach.  Uses the handle's segment store (as the adjoint does):
 * calls on one handle must not overlap. */
tpcfit_status tpcfit_smooth(tpcfit_handle* h, const tpcfit_hits* hits, const int32_t* track_offsets, int32_t n_tracks,
                            const int32_t* ndf, float* resid, float* rcov, float* chi2, void* stream);

/* Smoothed states of the recorded fit: for every cluster, the estimate of the
 * track state at that cluster from all the clusters of its track -- the
 * two-filter form of the smoother (Fraser & Potter), the outward pass's
 * filtered state at the cluster combined with the inward prediction there.
 * Inputs as for tpcfit_smooth (the last tpcfit_fit on this handle, with
 * recording on, same mode; otherwise ESTATE).  Outputs (device, overwritten):
 *   state:     float [n_hits][5], (y, z, sin phi, tan lambda, q/pt) at the
 *              cluster's pad row, in its sector's frame, y and z absolute;
 *   state_cov: float [n_hits][15], its covariance (packed lower-triangular).
 * NaN for the clusters of tracks with ndf <= 0 and for clusters the outward
 * pass did not reach.  Uses the handle's segment store: calls on one handle
 * must not overlap. */
tpcfit_status tpcfit_smooth_states(tpcfit_handle* h, const tpcfit_hits* hits, const int32_t* track_offsets,
                                   int32_t n_tracks, const int32_t* ndf, float* state, float* state_cov,
                                   void* stream);

/* Outlier rejection (the cluster-to-track association the smoother's chi2
 * tests; Sec. 2 keeps that relation's order deterministic): the clusters
 * whose leave-one-out chi2 from tpcfit_smooth is above chi2_cut are dropped
 * from their tracks, all others are copied, in their order, into
 * (y_out, z_out, rowsec_out).  offsets_out [n_tracks + 1] receives the new
 * track offsets; its last element is the number of clusters kept.  A cluster
 * whose chi2 is NaN (an unfitted track, a cluster the fit did not reach) is
 * kept.  The seeds stay as they were: a track whose first cluster is dropped
 * starts its refit from its old seed at the new first cluster's row, which the
 * diffuse start (100 cm^2, 100 in the angles and q/pt) makes immaterial for
 * all but the shortest tracks.  Inputs: the hits and offsets of the smoothed
 * fit (device) and its per-cluster chi2 (device float [n_hits]).  Outputs:
 * device arrays of n_hits elements (at most that many are written) and
 * offsets_out; they must not overlap the inputs.  Tracks whose offsets are
 * out of order or outside the arrays keep no cluster; tracks whose ranges
 * overlap give unspecified contents, and nothing is written beyond n_hits
 * elements.  Deterministic: the
 * result does not depend on the launch.  EINVAL for a negative or NaN cut,
 * missing or misaligned pointers, n_hits > INT32_MAX. */
tpcfit_status tpcfit_reject_outliers(tpcfit_handle* h, const tpcfit_hits* hits, const int32_t* track_offsets,
                                     int32_t n_tracks, const float* chi2, float chi2_cut, float* y_out, float* z_out,
                                     uint16_t* rowsec_out, int32_t* offsets_out, void* stream);

/* Fit + adjoint with HOST buffers, for streams of batches.  Copies hits,
 * offsets, seeds and grad_chi2 (host, as for tpcfit_fit and
 * tpcfit_fit_backward) to the device on an internal copy stream, fits with
 * recording on and runs the adjoint on `stream`, and copies back:
 *   chi2_out [n_tracks], ndf_out [n_tracks], grad_align_out [36][152][2],
 *   grad_seeds_out [5][n_tracks] (host).
 * Returns once the work is enqueued: the outputs are valid when `stream` has
 * passed this call (synchronise it, or an event recorded after the call), and
 * the inputs must stay unchanged until then.  The handle keeps two device
 * staging sets and uses them in turn, so the copies of the next call overlap
 * this call's fit and adjoint (with pinned host memory).  It leaves the
 * handle's recorded fit (for tpcfit_fit_backward and tpcfit_smooth) set to
 * this batch.  n_tracks = 0 zeroes grad_align_out and returns.  EINVAL for
 * missing pointers or n_hits above INT32_MAX. */
tpcfit_status tpcfit_fit_adjoint_host(tpcfit_handle* h, const float* y, const float* z, const uint16_t* rowsec,
                                      int64_t n_hits, const int32_t* track_offsets, int32_t n_tracks,
                                      const float* seeds, const float* grad_chi2, float* chi2_out, int32_t* ndf_out,
                                      float* grad_align_out, float* grad_seeds_out, void* stream);

/* Fit with HOST buffers: copies hits, offsets and seeds to the device, fits and
 * copies the outputs back, then synchronises `stream`.  Same argument meaning
 * as tpcfit_fit with every array in host memory (pinned memory gives
 * asynchronous copies).  The batch is streamed in chunks of about 196,608
 * tracks (at most 8): a chunk is copied on the library's copy stream while the
 * one before it is fitted on `stream`; results do not depend on the chunking.
 * With recording on (tpcfit_set_record) the batch is one chunk, since the
 * adjoint follows a single recorded fit.  EINVAL if the offsets at the chunk
 * boundaries decrease or exceed n_hits.  Device staging buffers are owned by
 * the handle and grown as needed. */
tpcfit_status tpcfit_fit_host(tpcfit_handle* h, const float* y, const float* z, const uint16_t* rowsec,
                              int64_t n_hits, const int32_t* track_offsets, int32_t n_tracks, const float* seeds,
                              float* params_out, float* cov_out, float* chi2_out, int32_t* ndf_out, void* stream);

/* Largest n_tracks that tpcfit_fit_noalloc accepts (2^20). */
#define TPCFIT_NOALLOC_MAX_TRACKS 1048576

/* Fit without allocating device memory and without a handle.
 * The paper has no counterpart; this entry point is for callers that cannot
 * call cudaMalloc or cudaFree: real-time loops that forbid allocator calls
 * (and the device synchronisation they can imply), or frameworks that only
 * hand out their own buffers.  It computes exactly what tpcfit_fit computes
 * with the default launch configuration (length ordering on, 4 rows per
 * stage, 24 warps per block), in the fast (deterministic = 0) or
 * deterministic (1) mode.
 *   geometry, bz_tesla: as for tpcfit_create; the constants are rebuilt on
 *               every call and travel in the launch's argument block, so no
 *               copy to the device is made for them and no other call (with
 *               or without a handle) sees them.
 *   alignment:  device float [36][152][2] offsets, or NULL for none.
 *   other arguments and outputs: as for tpcfit_fit.
 * Its scratch is a fixed static device array of about 4.3 MB (room for
 * TPCFIT_NOALLOC_MAX_TRACKS tracks) that each GPU loading the library holds
 * until the process exits; n_tracks above TPCFIT_NOALLOC_MAX_TRACKS returns
 * EINVAL without touching the GPU.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) and keeps it for the life of
 * the process; make that first call before any stream capture, and do not
 * call this entry point again on a device after cudaDeviceReset.  All calls
 * share the one array, so calls whose work overlaps on the GPU (other
 * streams, other host threads) race: serialise them.  Each call clears the
 * array's error word and work counter before its kernels run.  Invalid input
 * gives ndf = -2 and NaNs for the track (there is no error word to read
 * back); the other tracks of the call are unaffected. */
tpcfit_status tpcfit_fit_noalloc(const tpcfit_geometry* geometry, double bz_tesla, const float* alignment,
                                 int deterministic, const tpcfit_hits* hits, const int32_t* track_offsets,
                                 int32_t n_tracks, const float* seeds, float* params_out, float* cov_out,
                                 float* chi2_out, int32_t* ndf_out, void* stream);

/* Read (and clear) the handle's device error word: the first code a kernel
 * recorded (0 = none; 1 = bad offsets or frame table, 2 = row or sector out of
 * range, 3 = a frame-ready wait ran out) and the track it was found on (-1 if
 * none).  Synchronises `stream`.  Returns ETIMEOUT for code 3, EDEVICE for the
 * others, OK if nothing was recorded. */
tpcfit_status tpcfit_get_status(tpcfit_handle* h, void* stream, int32_t* err_code, int64_t* err_track);

/* FP32 throughput of this GPU, measured: the peak the fit's throughput is
 * reported against (the paper has no counterpart).  One launch of a kernel
 * that runs 8 independent FMA chains per thread, 2,048 threads on every SM,
 * `iterations` times 32 FMAs per chain; mode 0 scalar FMAs, mode 1 paired
 * fma.f32x2.  One short warm-up launch precedes it.  On return (the call
 * synchronises `stream`): *flop_out = the FP32 operations executed (an FMA
 * counts 2), *ms_out = the timed launch's duration from CUDA events on
 * `stream`.  EINVAL for another mode, iterations < 1 or a null output. */
tpcfit_status tpcfit_fp32_peak(int mode, int64_t iterations, void* stream, double* flop_out, double* ms_out);

/* Static description of a status code. */
const char* tpcfit_status_string(tpcfit_status s);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int32_t tpcfit_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TPCFIT_H_ */

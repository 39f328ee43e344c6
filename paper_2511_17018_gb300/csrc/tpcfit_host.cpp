// Host side of libtpcfit: the C ABI of include/tpcfit.h.  Validates arguments,
// owns the handle's device scratch, builds the per-time-frame constants (Sec.
// 4.1) that every launch carries in its argument block, and enqueues the
// kernels.
#include "tpcfit.h"

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

#include "internal.h"

namespace tpcfit {

bool backward_shape_supported(int warps) { return warps == 4 || warps == 8 || warps == 10 || warps == 12; }

bool fit_shape_supported(int lanes_per_track, int rows_per_stage, int warps) {
  if (lanes_per_track == 2 || lanes_per_track == 4 || lanes_per_track == 8 || lanes_per_track == 16 ||
      lanes_per_track == 32)
    return rows_per_stage == 4 && warps == 24;
  if (lanes_per_track != 1) return false;
  return (rows_per_stage == 4 && (warps == 8 || warps == 12 || warps == 24)) ||
         (rows_per_stage == 8 && (warps == 8 || warps == 16)) || (rows_per_stage == 16 && warps == 8);
}

// Build the per-time-frame constants on the host in FP64, rounded to FP32.
bool build_geo(const tpcfit_geometry* g, double bz, GeoConst& out) {
  if (!g || !g->row_x || g->n_sectors != kNSectors || g->n_rows < 1 || g->n_rows > kMaxRows) return false;
  // 18 sectors per side must cover the circle (the rotation table wraps at 9 sector steps)
  if (!(std::fabs(g->sector_width_deg * kNSide - 360.0) <= 1e-9) || !std::isfinite(bz)) return false;
  std::memset(&out, 0, sizeof(out));
  for (int r = 0; r < g->n_rows; ++r) {
    if (!std::isfinite(g->row_x[r]) || !(g->row_x[r] > 0.0)) return false;
    if (r > 0 && !(g->row_x[r] > g->row_x[r - 1])) return false;
    out.row_x[r] = (float)g->row_x[r];
  }
  // rotation from sector a to b: m = (b - a) mod 18 in [-8, 9], angle m * width
  const double w_rad = g->sector_width_deg * 3.14159265358979323846 / 180.0;
  for (int a = 0; a < kNSide; ++a)
    for (int b = 0; b < kNSide; ++b) {
      int m = ((b - a) % kNSide + kNSide) % kNSide;
      if (m > 9) m -= kNSide;
      const double da = (double)m * w_rad;
      out.rot_c[a * kNSide + b] = (float)std::cos(da);
      out.rot_s[a * kNSide + b] = (float)std::sin(da);
    }
  out.kappa = (float)(-0.00299792458 * bz);
  out.v_meas = (float)0.01;
  out.sqrt_v = (float)0.1;
  out.l0 = (float)std::sqrt((double)(float)100.0);
  out.max_snp = (float)0.999;
  out.n_rows = g->n_rows;
  return true;
}

}  // namespace tpcfit

using namespace tpcfit;

// tpcfit_fit_host streams a batch in chunks of about this many tracks (at
// most kHostChunksMax), copying one while the previous one is fitted.  A fit
// takes at least the time of its longest tracks (about 0.44 ms for 152-row
// tracks, whatever the batch size), so chunks stay large.
constexpr size_t kHostChunkTracks = 196608;
constexpr int kHostChunksMax = 8;

struct tpcfit_handle {
  int device = 0;
  GeoConst geo{};
  int deterministic = 0;
  int lanes_per_track = 1;
  int rows_per_stage = 4;
  int warps_per_block = 24;
  int sort_by_length = 1;
  float* d_align = nullptr;
  unsigned long long* d_err = nullptr;
  unsigned int* d_work = nullptr;
  int32_t* d_sort_scratch = nullptr;
  int32_t* d_perm = nullptr;
  int64_t perm_cap = 0;
  // staging for tpcfit_fit_host
  unsigned char* d_stage = nullptr;
  size_t stage_cap = 0;
  // tpcfit_fit_adjoint_host: two staging sets used in turn, their copy stream
  // and events (inputs copied; the set's last reader finished)
  unsigned char* d_pipe[2] = {nullptr, nullptr};
  size_t pipe_cap[2] = {0, 0};
  int pipe_slot = 0;
  cudaStream_t pipe_copy = nullptr;
  cudaEvent_t pipe_in[2] = {nullptr, nullptr};
  cudaEvent_t pipe_free[2] = {nullptr, nullptr};
  // tpcfit_fit_host: one event per chunk copied
  cudaEvent_t chunk_in[kHostChunksMax] = {};
  // adjoint: checkpoints of the last recorded fit
  int record = 0;
  int bwd_warps = 8;
  int bwd_form = 1;            // factor of the fast one-kernel backward: 1 U-D, 0 square root
  int det_reduce = 0;          // deterministic alignment gradient: 0 fixed-point sums, 1 key sort + fixed-order sums
  int fit_form = 1;            // factor of the fast fit without material: 1 U-D, 0 square root
  int rtc = 0;                 // fit kernels compiled at run time (Sec. 5)
  std::string rtc_dir;         // their on-disk cache, or empty
  float* d_ck = nullptr;
  int64_t ck_cap = 0;          // floats
  int32_t* d_ck_last = nullptr;
  int64_t ck_last_cap = 0;
  int64_t ck_slots = 0;
  bool rec_valid = false;
  int64_t rec_tracks = 0, rec_hits = 0;
  int rec_det = 0;
  int rec_form = 0;            // factor the recorded fit carried (1: U-D, its checkpoints hold U sqrt(D))
  // adjoint scratch: per-cluster gradients and the key sort
  float4* d_seg = nullptr;     // the segment store of the backward (fast mode) and the smoother
  int64_t seg_cap = 0;         // float4 elements
  float4* d_tape = nullptr;    // the backward's tape: the state before every step of both passes
  int64_t tape_cap = 0;        // float4 elements
  float* d_gm = nullptr;
  int64_t gm_cap = 0;          // floats
  unsigned char* d_keys = nullptr;
  size_t keys_cap = 0;
  // batched frames: ordering scratch
  int32_t* d_reject = nullptr;  // scan scratch of the outlier rejection
  int64_t reject_cap = 0;       // ints
  int32_t* d_frame_scratch = nullptr;
  int64_t frame_scratch_cap = 0;
};

namespace {

tpcfit_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return TPCFIT_OK;
  if (e == cudaErrorMemoryAllocation) return TPCFIT_ENOMEM;
  return TPCFIT_ECUDA;
}

bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

template <class T>
tpcfit_status grow(T*& ptr, int64_t& cap, int64_t need) {
  if (need <= cap) return TPCFIT_OK;
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  cap = 0;
  cudaError_t e = cudaMalloc(&ptr, sizeof(T) * (size_t)need);
  if (e != cudaSuccess) return from_cuda(e);
  cap = need;
  return TPCFIT_OK;
}

// Lazily created copy stream and events of the host-buffer entry points.
tpcfit_status ensure_pipe(tpcfit_handle* h) {
  if (h->pipe_copy) return TPCFIT_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&h->pipe_copy, cudaStreamNonBlocking);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
    e = cudaEventCreateWithFlags(&h->pipe_in[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->pipe_free[i], cudaEventDisableTiming);
  }
  for (int i = 0; i < kHostChunksMax && e == cudaSuccess; ++i)
    e = cudaEventCreateWithFlags(&h->chunk_in[i], cudaEventDisableTiming);
  return from_cuda(e);
}

tpcfit_status ensure_perm(tpcfit_handle* h, int64_t n) {
  if (n <= h->perm_cap) return TPCFIT_OK;
  if (h->d_perm) cudaFree(h->d_perm);
  h->d_perm = nullptr;
  h->perm_cap = 0;
  cudaError_t e = cudaMalloc(&h->d_perm, sizeof(int32_t) * (size_t)n);
  if (e != cudaSuccess) return from_cuda(e);
  h->perm_cap = n;
  return TPCFIT_OK;
}

}  // namespace

extern "C" {

int32_t tpcfit_version(void) { return 1 * 10000 + 0 * 100 + 0; }

namespace {
// The fit launch of a handle: ahead-of-time kernels, or the kernel compiled
// at run time for the handle's constants.
tpcfit_status launch_fit(const tpcfit_handle* h, const FitArgs& a, cudaStream_t s) {
  if (h->rtc && h->lanes_per_track == 1)
    return rtc_launch_fit(h->geo, h->deterministic != 0, h->rows_per_stage, h->warps_per_block, a,
                          h->rtc_dir.empty() ? nullptr : h->rtc_dir.c_str(), s);
  const cudaError_t e = h->deterministic
                            ? launch_fit_det(a, h->lanes_per_track, h->rows_per_stage, h->warps_per_block, s)
                            : launch_fit_fast(a, h->lanes_per_track, h->rows_per_stage, h->warps_per_block, s);
  return from_cuda(e);
}
}  // namespace

const char* tpcfit_status_string(tpcfit_status s) {
  switch (s) {
    case TPCFIT_OK: return "ok";
    case TPCFIT_EINVAL: return "invalid argument";
    case TPCFIT_ECUDA: return "CUDA runtime error";
    case TPCFIT_ENOMEM: return "device allocation failed";
    case TPCFIT_EDEVICE: return "a kernel found invalid input";
    case TPCFIT_ETIMEOUT: return "a bounded device-side wait ran out";
    case TPCFIT_ESTATE: return "call not allowed in the current state";
    case TPCFIT_ERTC: return "run-time compilation unavailable or failed";
  }
  return "unknown status";
}

tpcfit_status tpcfit_create(const tpcfit_geometry* geometry, double bz_tesla, tpcfit_handle** out) {
  if (!out) return TPCFIT_EINVAL;
  *out = nullptr;
  tpcfit_handle* h = new (std::nothrow) tpcfit_handle();
  if (!h) return TPCFIT_ENOMEM;
  if (!build_geo(geometry, bz_tesla, h->geo)) {
    delete h;
    return TPCFIT_EINVAL;
  }
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_align, sizeof(float) * kAlignFloats);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_err, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_work, sizeof(unsigned int) * 64);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_sort_scratch, sizeof(int32_t) * 512);
  if (e == cudaSuccess) e = cudaMemset(h->d_align, 0, sizeof(float) * kAlignFloats);
  if (e == cudaSuccess) e = cudaMemset(h->d_err, 0, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    tpcfit_destroy(h);
    return from_cuda(e);
  }
  *out = h;
  return TPCFIT_OK;
}

void tpcfit_destroy(tpcfit_handle* h) {
  if (!h) return;
  cudaDeviceSynchronize();
  if (h->d_align) cudaFree(h->d_align);
  if (h->d_err) cudaFree(h->d_err);
  if (h->d_work) cudaFree(h->d_work);
  if (h->d_sort_scratch) cudaFree(h->d_sort_scratch);
  if (h->d_perm) cudaFree(h->d_perm);
  if (h->d_stage) cudaFree(h->d_stage);
  for (int i = 0; i < 2; ++i) {
    if (h->d_pipe[i]) cudaFree(h->d_pipe[i]);
    if (h->pipe_in[i]) cudaEventDestroy(h->pipe_in[i]);
    if (h->pipe_free[i]) cudaEventDestroy(h->pipe_free[i]);
  }
  for (int i = 0; i < kHostChunksMax; ++i)
    if (h->chunk_in[i]) cudaEventDestroy(h->chunk_in[i]);
  if (h->pipe_copy) cudaStreamDestroy(h->pipe_copy);
  if (h->d_ck) cudaFree(h->d_ck);
  if (h->d_ck_last) cudaFree(h->d_ck_last);
  if (h->d_gm) cudaFree(h->d_gm);
  if (h->d_seg) cudaFree(h->d_seg);
  if (h->d_tape) cudaFree(h->d_tape);
  if (h->d_keys) cudaFree(h->d_keys);
  if (h->d_frame_scratch) cudaFree(h->d_frame_scratch);
  if (h->d_reject) cudaFree(h->d_reject);
  delete h;
}

tpcfit_status tpcfit_set_mode(tpcfit_handle* h, int deterministic) {
  if (!h || (deterministic != 0 && deterministic != 1)) return TPCFIT_EINVAL;
  h->deterministic = deterministic;
  return TPCFIT_OK;
}

tpcfit_status tpcfit_set_config(tpcfit_handle* h, int lanes_per_track, int rows_per_stage, int warps_per_block,
                                int sort_by_length) {
  if (!h) return TPCFIT_EINVAL;
  if (!fit_shape_supported(lanes_per_track, rows_per_stage, warps_per_block)) return TPCFIT_EINVAL;
  h->lanes_per_track = lanes_per_track;
  h->rows_per_stage = rows_per_stage;
  h->warps_per_block = warps_per_block;
  h->sort_by_length = sort_by_length ? 1 : 0;
  return TPCFIT_OK;
}

tpcfit_status tpcfit_set_alignment(tpcfit_handle* h, const float* d, void* stream) {
  if (!h) return TPCFIT_EINVAL;
  if (d && !aligned(d, 4)) return TPCFIT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = d ? cudaMemcpyAsync(h->d_align, d, sizeof(float) * kAlignFloats, cudaMemcpyDeviceToDevice, s)
                    : cudaMemsetAsync(h->d_align, 0, sizeof(float) * kAlignFloats, s);
  return from_cuda(e);
}

tpcfit_status tpcfit_reserve(tpcfit_handle* h, int64_t max_tracks, int64_t max_hits) {
  if (!h || max_tracks < 0 || max_hits < 0 || max_tracks > INT32_MAX) return TPCFIT_EINVAL;
  return ensure_perm(h, max_tracks);
}

tpcfit_status tpcfit_fit(tpcfit_handle* h, const tpcfit_hits* hits, const int32_t* track_offsets, int32_t n_tracks,
                         const float* seeds, float* params_out, float* cov_out, float* chi2_out, int32_t* ndf_out,
                         void* stream) {
  if (!h || !hits || n_tracks < 0 || hits->n_hits < 0) return TPCFIT_EINVAL;
  if (n_tracks == 0) return TPCFIT_OK;
  if (!track_offsets || !seeds || !params_out || !cov_out || !chi2_out || !ndf_out) return TPCFIT_EINVAL;
  if (hits->n_hits > 0 && (!hits->y || !hits->z || !hits->rowsec)) return TPCFIT_EINVAL;
  if (!aligned(hits->y, 4) || !aligned(hits->z, 4) || !aligned(hits->rowsec, 2) || !aligned(track_offsets, 4) ||
      !aligned(seeds, 4) || !aligned(params_out, 4) || !aligned(cov_out, 4) || !aligned(chi2_out, 4) ||
      !aligned(ndf_out, 4))
    return TPCFIT_EINVAL;
  if (hits->n_hits > INT32_MAX) return TPCFIT_EINVAL;  // int32 track offsets
  cudaStream_t s = (cudaStream_t)stream;
  tpcfit_status st = TPCFIT_OK;
  FitArgs a{};
  a.geo = h->geo;
  a.form = (!h->deterministic && !h->geo.mat) ? h->fit_form : 0;
  a.y = hits->y;
  a.z = hits->z;
  a.rowsec = hits->rowsec;
  a.n_hits = hits->n_hits;
  a.off = track_offsets;
  a.n_tracks = n_tracks;
  a.seeds = seeds;
  a.align = h->d_align;
  a.perm = nullptr;
  a.params = params_out;
  a.cov = cov_out;
  a.chi2 = chi2_out;
  a.ndf = ndf_out;
  a.err = h->d_err;
  a.work = h->d_work;
  a.mat = h->geo.mat;
  a.field = h->geo.field;
  h->rec_valid = false;
  if (h->record) {
    const int64_t slots = hits->n_hits / kCkptEvery + (int64_t)n_tracks + 1;
    st = grow(h->d_ck, h->ck_cap, 2 * slots * kCkptFloats);
    if (st == TPCFIT_OK) st = grow(h->d_ck_last, h->ck_last_cap, (int64_t)n_tracks);
    if (st != TPCFIT_OK) return st;
    a.ck = h->d_ck;
    a.ck_last = h->d_ck_last;
    a.ck_slots = slots;
    h->ck_slots = slots;
  }
  if (h->sort_by_length) {
    st = ensure_perm(h, n_tracks);
    if (st != TPCFIT_OK) return st;
    cudaError_t e = launch_length_order(track_offsets, n_tracks, h->d_perm, h->d_sort_scratch, s);
    if (e != cudaSuccess) return from_cuda(e);
    a.perm = h->d_perm;
  }
  st = launch_fit(h, a, s);
  if (st != TPCFIT_OK) return st;
  if (h->record) {
    h->rec_valid = true;
    h->rec_tracks = n_tracks;
    h->rec_hits = hits->n_hits;
    h->rec_det = h->deterministic;
    h->rec_form = (a.form == 1 && h->lanes_per_track == 1) ? 1 : 0;  // several lanes per track: square root
  }
  return TPCFIT_OK;
}

tpcfit_status tpcfit_fit_frames(tpcfit_handle* h, const tpcfit_hits* hits, const int32_t* track_offsets,
                                int32_t n_tracks, const int64_t* frame_track_base, int32_t n_frames,
                                const float* frame_alignment, const int32_t* frame_ready, int64_t wait_timeout_ns,
                                const float* seeds, float* params_out, float* cov_out, float* chi2_out,
                                int32_t* ndf_out, void* stream) {
  if (!h || !hits || n_tracks < 0 || hits->n_hits < 0 || n_frames < 1 || !frame_track_base) return TPCFIT_EINVAL;
  if (wait_timeout_ns < 0) return TPCFIT_EINVAL;
  if (n_tracks == 0) return TPCFIT_OK;
  if (!track_offsets || !seeds || !params_out || !cov_out || !chi2_out || !ndf_out) return TPCFIT_EINVAL;
  if (hits->n_hits > 0 && (!hits->y || !hits->z || !hits->rowsec)) return TPCFIT_EINVAL;
  if (!aligned(hits->y, 4) || !aligned(hits->z, 4) || !aligned(hits->rowsec, 2) || !aligned(track_offsets, 4) ||
      !aligned(seeds, 4) || !aligned(params_out, 4) || !aligned(cov_out, 4) || !aligned(chi2_out, 4) ||
      !aligned(ndf_out, 4) || !aligned(frame_track_base, 8) || (frame_alignment && !aligned(frame_alignment, 8)) ||
      (frame_ready && !aligned(frame_ready, 4)))
    return TPCFIT_EINVAL;
  if (hits->n_hits > INT32_MAX) return TPCFIT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  // ready flags are set by work on other streams; on the legacy default stream
  // that work would wait for the fit itself
  if (frame_ready && (s == nullptr || s == cudaStreamLegacy)) return TPCFIT_EINVAL;
  tpcfit_status st = ensure_perm(h, n_tracks);
  if (st == TPCFIT_OK) st = grow(h->d_frame_scratch, h->frame_scratch_cap, frame_order_scratch_ints(n_frames));
  if (st != TPCFIT_OK) return st;
  FitArgs a{};
  a.geo = h->geo;
  a.form = (!h->deterministic && !h->geo.mat) ? h->fit_form : 0;
  a.y = hits->y;
  a.z = hits->z;
  a.rowsec = hits->rowsec;
  a.n_hits = hits->n_hits;
  a.off = track_offsets;
  a.n_tracks = n_tracks;
  a.seeds = seeds;
  a.align = h->d_align;
  a.perm = h->d_perm;
  a.params = params_out;
  a.cov = cov_out;
  a.chi2 = chi2_out;
  a.ndf = ndf_out;
  a.err = h->d_err;
  a.work = h->d_work;
  a.mat = h->geo.mat;
  a.field = h->geo.field;
  a.frame_base = frame_track_base;
  a.n_frames = n_frames;
  a.frame_align = frame_alignment;
  a.frame_ready = frame_ready;
  a.wait_ns = wait_timeout_ns > 0 ? wait_timeout_ns : 1000000000LL;
  h->rec_valid = false;  // the adjoint follows single-frame fits only
  cudaError_t e =
      launch_frame_length_order(track_offsets, n_tracks, frame_track_base, n_frames, h->d_perm, h->d_frame_scratch, s);
  if (e != cudaSuccess) return from_cuda(e);
  return launch_fit(h, a, s);
}

tpcfit_status tpcfit_set_backward_config(tpcfit_handle* h, int warps_per_block) {
  if (!h || !backward_shape_supported(warps_per_block)) return TPCFIT_EINVAL;
  h->bwd_warps = warps_per_block;
  return TPCFIT_OK;
}

tpcfit_status tpcfit_reject_outliers(tpcfit_handle* h, const tpcfit_hits* hits, const int32_t* track_offsets,
                                     int32_t n_tracks, const float* chi2, float chi2_cut, float* y_out, float* z_out,
                                     uint16_t* rowsec_out, int32_t* offsets_out, void* stream) {
  if (!h || !hits || n_tracks < 0 || hits->n_hits < 0 || hits->n_hits > INT32_MAX || !offsets_out) return TPCFIT_EINVAL;
  if (!(chi2_cut >= 0.0f) || !aligned(offsets_out, 4)) return TPCFIT_EINVAL;  // a NaN cut is refused too
  if (n_tracks > 0 && (!track_offsets || !aligned(track_offsets, 4))) return TPCFIT_EINVAL;
  if (hits->n_hits > 0) {
    if (!hits->y || !hits->z || !hits->rowsec || !chi2 || !y_out || !z_out || !rowsec_out) return TPCFIT_EINVAL;
    if (!aligned(chi2, 4) || !aligned(y_out, 4) || !aligned(z_out, 4) || !aligned(rowsec_out, 2)) return TPCFIT_EINVAL;
  }
  tpcfit_status st = grow(h->d_reject, h->reject_cap, reject_scratch_ints(n_tracks));
  if (st != TPCFIT_OK) return st;
  return from_cuda(launch_reject(track_offsets, n_tracks, hits->y, hits->z, hits->rowsec, hits->n_hits, chi2,
                                 chi2_cut, y_out, z_out, rowsec_out, offsets_out, h->d_reject,
                                 (cudaStream_t)stream));
}

tpcfit_status tpcfit_set_fit_form(tpcfit_handle* h, int form) {
  if (!h || (form != 0 && form != 1)) return TPCFIT_EINVAL;
  h->fit_form = form;
  h->rec_valid = false;
  return TPCFIT_OK;
}

tpcfit_status tpcfit_set_det_reduction(tpcfit_handle* h, int method) {
  if (!h || (method != 0 && method != 1)) return TPCFIT_EINVAL;
  h->det_reduce = method;
  return TPCFIT_OK;
}

tpcfit_status tpcfit_set_backward_form(tpcfit_handle* h, int form) {
  if (!h || (form != 0 && form != 1)) return TPCFIT_EINVAL;
  h->bwd_form = form;
  return TPCFIT_OK;
}

tpcfit_status tpcfit_set_material(tpcfit_handle* h, double x0_cm, double dedx_gev_cm, double mass_gev,
                                  double row_cm) {
  if (!h) return TPCFIT_EINVAL;
  if (x0_cm <= 0.0) {  // no material
    h->geo.mat = 0;
    h->geo.x0_inv = h->geo.dedx = h->geo.mass2 = h->geo.d_row = 0.0f;
  } else {
    if (!std::isfinite(x0_cm) || !std::isfinite(dedx_gev_cm) || dedx_gev_cm < 0.0 || !(mass_gev > 0.0) ||
        !std::isfinite(mass_gev) || !(row_cm > 0.0) || !std::isfinite(row_cm))
      return TPCFIT_EINVAL;
    h->geo.mat = 1;
    h->geo.x0_inv = (float)(1.0 / x0_cm);
    h->geo.dedx = (float)dedx_gev_cm;
    h->geo.mass2 = (float)(mass_gev * mass_gev);
    h->geo.d_row = (float)row_cm;
  }
  h->rec_valid = false;
  return TPCFIT_OK;
}

tpcfit_status tpcfit_set_field_map(tpcfit_handle* h, double c_r, double c_z) {
  if (!h || !std::isfinite(c_r) || !std::isfinite(c_z)) return TPCFIT_EINVAL;
  h->geo.field = (c_r != 0.0 || c_z != 0.0) ? 1 : 0;
  h->geo.f_r = (float)(c_r / (250.0 * 250.0));
  h->geo.f_z = (float)(c_z / (250.0 * 250.0));
  h->rec_valid = false;
  return TPCFIT_OK;
}

tpcfit_status tpcfit_set_rtc(tpcfit_handle* h, int enable, const char* cache_dir) {
  if (!h || (enable != 0 && enable != 1)) return TPCFIT_EINVAL;
  if (enable && !rtc_available()) return TPCFIT_ERTC;
  h->rtc = enable;
  h->rtc_dir = cache_dir ? cache_dir : "";
  return TPCFIT_OK;
}

tpcfit_status tpcfit_rtc_build(const tpcfit_geometry* geometry, double bz_tesla, int deterministic, int rows_per_stage,
                               int warps_per_block, int record, int frames, const char* cache_dir) {
  GeoConst g{};
  if (!geometry || !build_geo(geometry, bz_tesla, g)) return TPCFIT_EINVAL;
  if (!fit_shape_supported(1, rows_per_stage, warps_per_block)) return TPCFIT_EINVAL;
  return rtc_build(g, deterministic != 0, rows_per_stage, warps_per_block, record != 0, frames != 0, cache_dir);
}

int tpcfit_rtc_available(void) { return rtc_available() ? 1 : 0; }
long long tpcfit_rtc_compile_count(void) { return rtc_compile_count(); }
const char* tpcfit_rtc_log(void) { return rtc_log(); }

tpcfit_status tpcfit_set_record(tpcfit_handle* h, int record) {
  if (!h || (record != 0 && record != 1)) return TPCFIT_EINVAL;
  h->record = record;
  if (!record) h->rec_valid = false;
  return TPCFIT_OK;
}

tpcfit_status tpcfit_fit_backward(tpcfit_handle* h, const tpcfit_hits* hits, const int32_t* track_offsets,
                                  int32_t n_tracks, const int32_t* ndf, const float* grad_chi2, float* grad_align,
                                  float* grad_seeds, float* grad_meas, void* stream) {
  if (!h || !hits || n_tracks < 0 || hits->n_hits < 0) return TPCFIT_EINVAL;
  if (!grad_align || !aligned(grad_align, 4)) return TPCFIT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  if (n_tracks == 0) return from_cuda(cudaMemsetAsync(grad_align, 0, sizeof(float) * kAlignFloats, s));
  if (!track_offsets || !ndf || !grad_chi2 || !grad_seeds) return TPCFIT_EINVAL;
  if (hits->n_hits > 0 && (!hits->y || !hits->z || !hits->rowsec)) return TPCFIT_EINVAL;
  if (!aligned(grad_chi2, 4) || !aligned(grad_seeds, 4) || !aligned(ndf, 4) || (grad_meas && !aligned(grad_meas, 8)))
    return TPCFIT_EINVAL;
  if (!h->rec_valid || h->rec_tracks != n_tracks || h->rec_hits != hits->n_hits ||
      h->rec_det != h->deterministic)
    return TPCFIT_ESTATE;
  tpcfit_status st = TPCFIT_OK;
  BwdArgs b{};
  b.geo = h->geo;
  b.y = hits->y;
  b.z = hits->z;
  b.rowsec = hits->rowsec;
  b.n_hits = hits->n_hits;
  b.off = track_offsets;
  b.n_tracks = n_tracks;
  b.align = h->d_align;
  b.perm = h->sort_by_length ? h->d_perm : nullptr;
  b.ndf = ndf;
  b.ck = h->d_ck;
  b.ck_last = h->d_ck_last;
  b.ck_slots = h->ck_slots;
  b.grad_chi2 = grad_chi2;
  b.grad_seeds = grad_seeds;
  b.work = h->d_work;
  b.phys = (h->geo.mat ? 1 : 0) | (h->geo.field ? 2 : 0);
  b.ck_form = h->rec_form;
  cudaError_t e = cudaSuccess;
  if (h->deterministic || h->geo.mat) {
    // where the forward step is expensive (no FMA; the material folding) the
    // backward replays the segments in a kernel of its own at the fit's
    // occupancy onto a tape (the state before every step of both passes, 152
    // steps per 32-track work item) and reverses from it; measured on 400k
    // tracks: deterministic 8.0 ms against 9.5 ms, material 7.0 against 9.4
    st = grow(h->d_tape, h->tape_cap, backward_tape_float4s(n_tracks));
    if (st != TPCFIT_OK) return st;
    b.tape = h->d_tape;
  } else {
    // otherwise one kernel recomputes each segment into a per-warp segment
    // store that stays in L2 until the reverse reads it back (square-root
    // factor: 4.7 ms against 5.6 ms with the tape)
    int64_t need = 0;
    // the square-root reverse hands each segment's factor adjoint to the
    // segment before it, which holds only if its recomputation reproduces the
    // recorded factor: after a U-D fit only the U-D reverse applies (the U-D
    // factorisation of a covariance is unique)
    if (h->bwd_form == 0 && h->rec_form == 1) return TPCFIT_ESTATE;
    b.form = h->bwd_form;
    e = backward_store_fast(h->bwd_warps, b.phys, b.form, need);
    if (e != cudaSuccess) return from_cuda(e);
    st = grow(h->d_seg, h->seg_cap, need);
    if (st != TPCFIT_OK) return st;
    b.seg = h->d_seg;
  }
  if (!h->deterministic) {
    // fast: atomics straight into the alignment gradient
    b.grad_meas = grad_meas;
    b.grad_align_atomic = grad_align;
    e = cudaMemsetAsync(grad_align, 0, sizeof(float) * kAlignFloats, s);
    if (e == cudaSuccess) e = launch_backward_fast(b, h->bwd_warps, s);
    return from_cuda(e);
  }
  // deterministic: per-cluster gradients, then a stable key sort and
  // fixed-order sums per key
  float* gm = grad_meas;
  if (!gm) {
    st = grow(h->d_gm, h->gm_cap, 2 * hits->n_hits);
    if (st != TPCFIT_OK) return st;
    gm = h->d_gm;
  }
  const size_t kb = h->det_reduce == 1 ? key_sort_scratch_bytes(hits->n_hits) : key_fixed_scratch_bytes();
  if (kb > h->keys_cap) {
    if (h->d_keys) cudaFree(h->d_keys);
    h->d_keys = nullptr;
    h->keys_cap = 0;
    e = cudaMalloc(&h->d_keys, kb);
    if (e != cudaSuccess) return from_cuda(e);
    h->keys_cap = kb;
  }
  b.grad_meas = gm;
  b.grad_align_atomic = nullptr;
  e = launch_backward_det(b, h->bwd_warps, s);
  if (h->det_reduce == 0) {
    if (e == cudaSuccess)
      e = launch_key_fixed_reduce(gm, hits->rowsec, hits->n_hits, h->geo.n_rows, h->d_keys, grad_align, s);
    return from_cuda(e);
  }
  int* sorted = nullptr;
  int* key_start = nullptr;
  if (e == cudaSuccess) e = launch_key_sort(hits->rowsec, hits->n_hits, h->geo.n_rows, h->d_keys, &sorted, &key_start, s);
  if (e == cudaSuccess) e = launch_key_reduce(gm, sorted, key_start, grad_align, s);
  return from_cuda(e);
}

namespace {
// The smoother of the recorded fit: the leave-one-out outputs (resid, rcov,
// chi2) and / or the smoothed states (state, state_cov); null pointers skip.
tpcfit_status run_smooth(tpcfit_handle* h, const tpcfit_hits* hits, const int32_t* track_offsets, int32_t n_tracks,
                         const int32_t* ndf, float* resid, float* rcov, float* chi2, float* state, float* state_cov,
                         void* stream) {
  if (!h || !hits || n_tracks < 0 || hits->n_hits < 0) return TPCFIT_EINVAL;
  if (n_tracks == 0) return TPCFIT_OK;
  if (!track_offsets || !ndf) return TPCFIT_EINVAL;
  if (hits->n_hits > 0 && (!hits->y || !hits->z || !hits->rowsec)) return TPCFIT_EINVAL;
  if (!aligned(ndf, 4) || (resid && (!aligned(resid, 8) || !aligned(rcov, 4) || !aligned(chi2, 4))) ||
      (state && (!aligned(state, 4) || !aligned(state_cov, 4))))
    return TPCFIT_EINVAL;
  if (!h->rec_valid || h->rec_tracks != n_tracks || h->rec_hits != hits->n_hits ||
      h->rec_det != h->deterministic)
    return TPCFIT_ESTATE;
  cudaStream_t s = (cudaStream_t)stream;
  tpcfit_status st = TPCFIT_OK;
  SmoothArgs a{};
  a.geo = h->geo;
  a.y = hits->y;
  a.z = hits->z;
  a.rowsec = hits->rowsec;
  a.n_hits = hits->n_hits;
  a.off = track_offsets;
  a.n_tracks = n_tracks;
  a.align = h->d_align;
  a.perm = h->sort_by_length ? h->d_perm : nullptr;
  a.ndf = ndf;
  a.ck = h->d_ck;
  a.ck_last = h->d_ck_last;
  a.ck_slots = h->ck_slots;
  a.resid = resid;
  a.rcov = rcov;
  a.chi2 = chi2;
  a.state = state;
  a.state_cov = state_cov;
  a.work = h->d_work;
  a.mat = h->geo.mat;
  a.ck_form = h->rec_form;
  int64_t need = 0;
  cudaError_t e = h->deterministic ? smooth_store_det(need) : smooth_store_fast(need);
  if (e != cudaSuccess) return from_cuda(e);
  st = grow(h->d_seg, h->seg_cap, need);
  if (st != TPCFIT_OK) return st;
  a.seg = h->d_seg;
  e = h->deterministic ? launch_smooth_det(a, s) : launch_smooth_fast(a, s);
  return from_cuda(e);
}
}  // namespace

tpcfit_status tpcfit_smooth(tpcfit_handle* h, const tpcfit_hits* hits, const int32_t* track_offsets, int32_t n_tracks,
                            const int32_t* ndf, float* resid, float* rcov, float* chi2, void* stream) {
  if (n_tracks > 0 && (!resid || !rcov || !chi2)) return TPCFIT_EINVAL;
  return run_smooth(h, hits, track_offsets, n_tracks, ndf, resid, rcov, chi2, nullptr, nullptr, stream);
}

tpcfit_status tpcfit_smooth_states(tpcfit_handle* h, const tpcfit_hits* hits, const int32_t* track_offsets,
                                   int32_t n_tracks, const int32_t* ndf, float* state, float* state_cov,
                                   void* stream) {
  if (n_tracks > 0 && (!state || !state_cov)) return TPCFIT_EINVAL;
  return run_smooth(h, hits, track_offsets, n_tracks, ndf, nullptr, nullptr, nullptr, state, state_cov, stream);
}

tpcfit_status tpcfit_fit_host(tpcfit_handle* h, const float* y, const float* z, const uint16_t* rowsec,
                              int64_t n_hits, const int32_t* track_offsets, int32_t n_tracks, const float* seeds,
                              float* params_out, float* cov_out, float* chi2_out, int32_t* ndf_out, void* stream) {
  if (!h || n_tracks < 0 || n_hits < 0 || n_hits > INT32_MAX) return TPCFIT_EINVAL;
  if (n_tracks == 0) return TPCFIT_OK;
  if (!track_offsets || !seeds || !params_out || !cov_out || !chi2_out || !ndf_out) return TPCFIT_EINVAL;
  if (n_hits > 0 && (!y || !z || !rowsec)) return TPCFIT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t N = (size_t)n_tracks, H = (size_t)n_hits;
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  // hits and offsets at their own positions; seeds and outputs per chunk,
  // [rows][chunk tracks] at the chunk's first track (rows x track offset)
  const size_t o_y = 0, o_z = o_y + up(4 * H), o_rs = o_z + up(4 * H), o_off = o_rs + up(2 * H),
               o_seed = o_off + up(4 * (N + 1)), o_par = o_seed + up(20 * N), o_cov = o_par + up(20 * N),
               o_chi = o_cov + up(60 * N), o_ndf = o_chi + up(4 * N), total = o_ndf + up(4 * N);
  if (total > h->stage_cap) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return from_cuda(e);
    if (h->d_stage) cudaFree(h->d_stage);
    h->d_stage = nullptr;
    h->stage_cap = 0;
    e = cudaMalloc(&h->d_stage, total);
    if (e != cudaSuccess) return from_cuda(e);
    h->stage_cap = total;
  }
  tpcfit_status st = ensure_pipe(h);
  if (st != TPCFIT_OK) return st;
  unsigned char* b = h->d_stage;
  // chunks of about kHostChunkTracks tracks; one chunk while recording, since
  // the adjoint follows a single recorded fit
  int K = (int)((N + kHostChunkTracks - 1) / kHostChunkTracks);
  if (K > kHostChunksMax) K = kHostChunksMax;
  if (K < 1 || h->record) K = 1;
  // the copies use the offsets at the chunk boundaries: they must be in order
  // and within the hits (the kernels check every track's offsets)
  for (int k = 0; k <= K; ++k) {
    const int32_t o = track_offsets[N * (size_t)k / (size_t)K];
    const int32_t prev = k ? track_offsets[N * (size_t)(k - 1) / (size_t)K] : 0;
    if (o < prev || (int64_t)o > n_hits) return TPCFIT_EINVAL;
  }
  cudaStream_t c = h->pipe_copy;
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < K && e == cudaSuccess; ++k) {
    const size_t t0 = N * (size_t)k / (size_t)K, t1 = N * (size_t)(k + 1) / (size_t)K, n = t1 - t0;
    const size_t h0 = (size_t)track_offsets[t0], h1 = (size_t)track_offsets[t1];
    if (h1 > h0) {
      e = cudaMemcpyAsync(b + o_y + 4 * h0, y + h0, 4 * (h1 - h0), cudaMemcpyHostToDevice, c);
      if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_z + 4 * h0, z + h0, 4 * (h1 - h0), cudaMemcpyHostToDevice, c);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(b + o_rs + 2 * h0, rowsec + h0, 2 * (h1 - h0), cudaMemcpyHostToDevice, c);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b + o_off + 4 * t0, track_offsets + t0, 4 * (n + 1), cudaMemcpyHostToDevice, c);
    // seeds [5][N] on the host -> [5][n] for the chunk
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(b + o_seed + 20 * t0, 4 * n, seeds + t0, 4 * N, 4 * n, 5, cudaMemcpyHostToDevice, c);
    if (e == cudaSuccess) e = cudaEventRecord(h->chunk_in[k], c);
  }
  if (e != cudaSuccess) return from_cuda(e);
  tpcfit_hits hh{(const float*)(b + o_y), (const float*)(b + o_z), (const uint16_t*)(b + o_rs), n_hits};
  for (int k = 0; k < K; ++k) {
    const size_t t0 = N * (size_t)k / (size_t)K, t1 = N * (size_t)(k + 1) / (size_t)K, n = t1 - t0;
    e = cudaStreamWaitEvent(s, h->chunk_in[k], 0);
    if (e != cudaSuccess) return from_cuda(e);
    float* par = (float*)(b + o_par + 20 * t0);
    float* cov = (float*)(b + o_cov + 60 * t0);
    st = tpcfit_fit(h, &hh, (const int32_t*)(b + o_off + 4 * t0), (int32_t)n, (const float*)(b + o_seed + 20 * t0),
                    par, cov, (float*)(b + o_chi) + t0, (int32_t*)(b + o_ndf) + t0, stream);
    if (st != TPCFIT_OK) return st;
    // [rows][n] -> the caller's [rows][N] at column t0
    e = cudaMemcpy2DAsync(params_out + t0, 4 * N, par, 4 * n, 4 * n, 5, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpy2DAsync(cov_out + t0, 4 * N, cov, 4 * n, 4 * n, 15, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(chi2_out + t0, (float*)(b + o_chi) + t0, 4 * n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(ndf_out + t0, (int32_t*)(b + o_ndf) + t0, 4 * n, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return from_cuda(e);
  }
  return from_cuda(cudaStreamSynchronize(s));
}

tpcfit_status tpcfit_fit_adjoint_host(tpcfit_handle* h, const float* y, const float* z, const uint16_t* rowsec,
                                      int64_t n_hits, const int32_t* track_offsets, int32_t n_tracks,
                                      const float* seeds, const float* grad_chi2, float* chi2_out, int32_t* ndf_out,
                                      float* grad_align_out, float* grad_seeds_out, void* stream) {
  if (!h || n_tracks < 0 || n_hits < 0 || n_hits > INT32_MAX) return TPCFIT_EINVAL;
  if (!grad_align_out) return TPCFIT_EINVAL;
  if (n_tracks > 0 && (!track_offsets || !seeds || !grad_chi2 || !chi2_out || !ndf_out || !grad_seeds_out))
    return TPCFIT_EINVAL;
  if (n_hits > 0 && (!y || !z || !rowsec)) return TPCFIT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (n_tracks == 0) {
    std::memset(grad_align_out, 0, sizeof(float) * kAlignFloats);
    return TPCFIT_OK;
  }
  const size_t N = (size_t)n_tracks, H = (size_t)n_hits;
  auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t o_y = 0, o_z = o_y + up(4 * H), o_rs = o_z + up(4 * H), o_off = o_rs + up(2 * H),
               o_seed = o_off + up(4 * (N + 1)), o_g = o_seed + up(20 * N), o_par = o_g + up(4 * N),
               o_cov = o_par + up(20 * N), o_chi = o_cov + up(60 * N), o_ndf = o_chi + up(4 * N),
               o_gs = o_ndf + up(4 * N), o_ga = o_gs + up(20 * N), total = o_ga + up(4 * (size_t)kAlignFloats);
  {
    tpcfit_status sp = ensure_pipe(h);
    if (sp != TPCFIT_OK) return sp;
  }
  const int slot = h->pipe_slot;
  if (total > h->pipe_cap[slot]) {
    // the set may still be in use by an earlier call's work (its readback included)
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return from_cuda(e);
    if (h->d_pipe[slot]) cudaFree(h->d_pipe[slot]);
    h->d_pipe[slot] = nullptr;
    h->pipe_cap[slot] = 0;
    e = cudaMalloc(&h->d_pipe[slot], total);
    if (e != cudaSuccess) return from_cuda(e);
    h->pipe_cap[slot] = total;
  }
  unsigned char* b = h->d_pipe[slot];
  // inputs, on the copy stream, once the set's previous reader has finished
  cudaStream_t c = h->pipe_copy;
  e = cudaStreamWaitEvent(c, h->pipe_free[slot], 0);
  if (e == cudaSuccess && H) e = cudaMemcpyAsync(b + o_y, y, 4 * H, cudaMemcpyHostToDevice, c);
  if (e == cudaSuccess && H) e = cudaMemcpyAsync(b + o_z, z, 4 * H, cudaMemcpyHostToDevice, c);
  if (e == cudaSuccess && H) e = cudaMemcpyAsync(b + o_rs, rowsec, 2 * H, cudaMemcpyHostToDevice, c);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_off, track_offsets, 4 * (N + 1), cudaMemcpyHostToDevice, c);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_seed, seeds, 20 * N, cudaMemcpyHostToDevice, c);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b + o_g, grad_chi2, 4 * N, cudaMemcpyHostToDevice, c);
  if (e == cudaSuccess) e = cudaEventRecord(h->pipe_in[slot], c);
  // fit with checkpoints and adjoint on the caller's stream
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->pipe_in[slot], 0);
  if (e != cudaSuccess) return from_cuda(e);
  h->pipe_slot = slot ^ 1;
  tpcfit_hits hh{(const float*)(b + o_y), (const float*)(b + o_z), (const uint16_t*)(b + o_rs), n_hits};
  const int rec = h->record;
  h->record = 1;
  tpcfit_status st = tpcfit_fit(h, &hh, (const int32_t*)(b + o_off), n_tracks, (const float*)(b + o_seed),
                                (float*)(b + o_par), (float*)(b + o_cov), (float*)(b + o_chi), (int32_t*)(b + o_ndf),
                                stream);
  h->record = rec;
  if (st == TPCFIT_OK)
    st = tpcfit_fit_backward(h, &hh, (const int32_t*)(b + o_off), n_tracks, (const int32_t*)(b + o_ndf),
                             (const float*)(b + o_g), (float*)(b + o_ga), (float*)(b + o_gs), nullptr, stream);
  if (st != TPCFIT_OK) return st;
  e = cudaEventRecord(h->pipe_free[slot], s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(chi2_out, b + o_chi, 4 * N, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ndf_out, b + o_ndf, 4 * N, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(grad_seeds_out, b + o_gs, 20 * N, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(grad_align_out, b + o_ga, sizeof(float) * kAlignFloats, cudaMemcpyDeviceToHost, s);
  return from_cuda(e);
}

tpcfit_status tpcfit_get_status(tpcfit_handle* h, void* stream, int32_t* err_code, int64_t* err_track) {
  if (!h) return TPCFIT_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long w = 0;
  cudaError_t e = cudaMemcpyAsync(&w, h->d_err, sizeof(w), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_err, 0, sizeof(w), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return from_cuda(e);
  const int32_t code = (int32_t)(w >> 56);
  if (err_code) *err_code = code;
  if (err_track) *err_track = code ? (int64_t)(w & 0x00FFFFFFFFFFFFFFull) : -1;
  if (code == (int32_t)kErrTimeout) return TPCFIT_ETIMEOUT;
  return code ? TPCFIT_EDEVICE : TPCFIT_OK;
}

}  // extern "C"
